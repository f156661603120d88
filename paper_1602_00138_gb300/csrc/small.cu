// Small dense float64 kernels: Cholesky of the Galerkin matrices V^T A~ V
// and of the per-RHS deflation matrices U_j^T A~ U_j, bordered Cholesky
// updates after a one-column append, batched triangular solves, the ordered
// rank-revealing Cholesky of the append (pivot-free, in candidate order,
// with a drop test) and a cyclic Jacobi eigensolver for Rayleigh-Ritz.
//
// All matrices are column-major; a Cholesky factor L is lower triangular.
// These run on one CTA (or one CTA per independent system): the matrices
// are at most a few thousand wide and live in global memory / L2.
#include "common.cuh"
#include "../../include/rcg.h"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

namespace rcg {
namespace {

__device__ __forceinline__ bool bad(double d) { return !(d > 0.0) || !isfinite(d); }

// Right-looking Cholesky of the lower triangle of A (r x r), steps k0..r-1.
// Columns < k0 must already be factored and applied to the trailing part.
__global__ void __launch_bounds__(1024) k_chol(double *A, int lda, int k0, int r, int *info) {
    __shared__ double piv;
    __shared__ int fail;
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    for (int k = k0; k < r; ++k) {
        if (threadIdx.x == 0) {
            const double d = A[k + (long long)k * lda];
            if (bad(d)) { fail = k + 1; }
            else { piv = sqrt(d); A[k + (long long)k * lda] = piv; }
        }
        __syncthreads();
        if (fail) break;
        const double inv = 1.0 / piv;
        for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) A[i + (long long)k * lda] *= inv;
        __syncthreads();
        const int m = r - k - 1;
        const long long tot = (long long)m * m;
        for (long long e = threadIdx.x; e < tot; e += blockDim.x) {
            const int ii = (int)(e % m), jj = (int)(e / m);
            if (ii < jj) continue;
            const int i = k + 1 + ii, j = k + 1 + jj;
            A[i + (long long)j * lda] -= A[i + (long long)k * lda] * A[j + (long long)k * lda];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && info && fail) atomicMax(info, fail);
}

// The same factorisation with the lower triangle staged in shared memory
// (r x r, ld r; r <= SM_R), for matrix b = blockIdx.x at A + b strideA: the
// r sequential steps then touch only shared memory.  Warp w updates trailing
// columns w, w + nw, ...; failure (first bad pivot + 1) goes to *info by
// atomicMax.
constexpr int SM_R = 160;
__global__ void __launch_bounds__(1024) k_chol_sm(double *A, int lda, long long strideA, int k0, int r, int *info) {
    extern __shared__ double S[];
    __shared__ double piv;
    __shared__ int fail;
    A += blockIdx.x * strideA;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = warp; j < r; j += nw)
        for (int i = j + lane; i < r; i += 32) S[i + j * r] = A[i + (long long)j * lda];
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    for (int k = k0; k < r; ++k) {
        if (threadIdx.x == 0) {
            const double d = S[k + k * r];
            if (bad(d)) fail = k + 1;
            else { piv = sqrt(d); S[k + k * r] = piv; }
        }
        __syncthreads();
        if (fail) break;
        const double inv = 1.0 / piv;
        for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) S[i + k * r] *= inv;
        __syncthreads();
        for (int j = k + 1 + warp; j < r; j += nw) {
            const double ljk = S[j + k * r];
            for (int i = j + lane; i < r; i += 32) S[i + j * r] -= S[i + k * r] * ljk;
        }
        __syncthreads();
    }
    for (int j = warp; j < r; j += nw)
        for (int i = j + lane; i < r; i += 32) A[i + (long long)j * lda] = S[i + j * r];
    if (threadIdx.x == 0 && info && fail) atomicMax(info, fail);
}

// New rows r_old..r_old+a-1 of A hold the Gram entries (lower part).  Apply
// the factored columns 0..r_old-1 to them (forward substitution), then the
// caller continues with k_chol(k0 = r_old).
__global__ void __launch_bounds__(1024) k_chol_border(double *A, int lda, int r_old, int a) {
    const int rn = r_old + a;
    for (int j = 0; j < r_old; ++j) {
        const double ljj = A[j + (long long)j * lda];
        for (int i = r_old + threadIdx.x; i < rn; i += blockDim.x) A[i + (long long)j * lda] /= ljj;
        __syncthreads();
        // rows i (new) : A[i][k] -= L[k][j] * L[i][j] for j < k < r_old,
        // and the new block A[i][k] for r_old <= k <= i
        const int m = rn - (j + 1);
        const long long tot = (long long)a * m;
        for (long long e = threadIdx.x; e < tot; e += blockDim.x) {
            const int i = r_old + (int)(e % a);
            const int k = j + 1 + (int)(e / a);
            if (k > i) continue;
            A[i + (long long)k * lda] -= A[k + (long long)j * lda] * A[i + (long long)j * lda];
        }
        __syncthreads();
    }
}

// Solve L y = b (or L^T y = b) for column blockIdx.x of B, in place.
__global__ void __launch_bounds__(256) k_trsv(const double *L, int ldl, int r, double *B, int ldb, int trans) {
    extern __shared__ double y[];
    double *b = B + (long long)blockIdx.x * ldb;
    for (int i = threadIdx.x; i < r; i += blockDim.x) y[i] = b[i];
    __syncthreads();
    if (!trans) {
        for (int j = 0; j < r; ++j) {
            const double yj = y[j] / L[j + (long long)j * ldl];
            __syncthreads();
            if (threadIdx.x == 0) y[j] = yj;
            for (int k = j + 1 + threadIdx.x; k < r; k += blockDim.x) y[k] -= L[k + (long long)j * ldl] * yj;
            __syncthreads();
        }
    } else {
        for (int j = r - 1; j >= 0; --j) {
            const double yj = y[j] / L[j + (long long)j * ldl];
            __syncthreads();
            if (threadIdx.x == 0) y[j] = yj;
            for (int k = threadIdx.x; k < j; k += blockDim.x) y[k] -= L[j + (long long)k * ldl] * yj;
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < r; i += blockDim.x) b[i] = y[i];
}

// Batched triangular solves with L staged in shared memory (r <= SM_R):
// system b = blockIdx.y has factor L + b strideL and right-hand sides
// B + b strideB; warp w of CTA blockIdx.x solves column 8 blockIdx.x + w in
// place (forward L y = b, or backward L^T y = b), synchronising only itself.
// The diagonal's reciprocals are formed once per CTA.
__global__ void __launch_bounds__(256) k_trsv_sm(const double *L, int ldl, long long strideL, int r, double *B,
                                                 int ldb, long long strideB, int m, int trans) {
    extern __shared__ double sh[];
    double *Ls = sh, *dinv = sh + (long long)r * r, *ys = dinv + r;
    L += blockIdx.y * strideL;
    B += blockIdx.y * strideB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = warp; j < r; j += 8)
        for (int i = j + lane; i < r; i += 32) Ls[i + j * r] = L[i + (long long)j * ldl];
    __syncthreads();
    for (int j = threadIdx.x; j < r; j += blockDim.x) dinv[j] = 1.0 / Ls[j + j * r];
    const int col = blockIdx.x * 8 + warp;
    double *y = ys + warp * r;
    double *b = B + (long long)col * ldb;
    if (col < m)
        for (int i = lane; i < r; i += 32) y[i] = b[i];
    __syncthreads();
    if (col >= m) return;
    if (!trans) {
        for (int j = 0; j < r; ++j) {
            const double yj = y[j] * dinv[j];
            __syncwarp();
            if (lane == 0) y[j] = yj;
            for (int k = j + 1 + lane; k < r; k += 32) y[k] -= Ls[k + j * r] * yj;
            __syncwarp();
        }
    } else {
        for (int j = r - 1; j >= 0; --j) {
            const double yj = y[j] * dinv[j];
            __syncwarp();
            if (lane == 0) y[j] = yj;
            for (int k = lane; k < j; k += 32) y[k] -= Ls[j + k * r] * yj;
            __syncwarp();
        }
    }
    for (int i = lane; i < r; i += 32) b[i] = y[i];
}

// Ordered pivot-free Cholesky of the candidate Gram M (a x a) with drop test:
// candidate c is kept iff its component orthogonal to the kept candidates
// before it, ||.||, divided by ||x_c||, exceeds tau.  R is upper triangular
// (row c = kept candidate c), S is scratch (a x a).
__global__ void __launch_bounds__(1024)
k_ordered_drop(const double *M, int a, const double *xnorm2, double tau, double *S, double *R, int *kept,
               double *ratio) {
    // S holds the trailing Schur complement; only its upper triangle (i <= j)
    // is kept up to date.  Row c of R is staged in shared memory.
    extern __shared__ double rowc[];
    __shared__ double piv;
    __shared__ int keep;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = warp; j < a; j += nw)
        for (int i = lane; i < a; i += 32) {
            S[i + (long long)j * a] = M[i + (long long)j * a];
            R[i + (long long)j * a] = 0.0;
        }
    __syncthreads();
    for (int c = 0; c < a; ++c) {
        if (threadIdx.x == 0) {
            const double d = S[c + (long long)c * a];
            const double rt = (d > 0.0 && isfinite(d)) ? sqrt(d / xnorm2[c]) : 0.0;
            ratio[c] = rt;
            keep = (rt > tau) ? 1 : 0;
            kept[c] = keep;
            piv = keep ? sqrt(d) : 0.0;
            if (keep) R[c + (long long)c * a] = piv;
        }
        __syncthreads();
        if (keep) {
            for (int j = c + 1 + threadIdx.x; j < a; j += blockDim.x) {
                const double v = S[c + (long long)j * a] / piv;
                R[c + (long long)j * a] = v;
                rowc[j] = v;
            }
            __syncthreads();
            // S(i, j) -= R(c, i) R(c, j) for c < i <= j: warps over columns, lanes over rows
            for (int j = c + 1 + warp; j < a; j += nw) {
                const double rj = rowc[j];
                for (int i = c + 1 + lane; i <= j; i += 32) S[i + (long long)j * a] -= rowc[i] * rj;
            }
        }
        __syncthreads();
    }
}

// Inverse of an upper triangular a x a matrix R (ld ldr) into Ri (ld a):
// thread j solves R x = e_j by back substitution.
__global__ void k_tri_upper_inv(const double *R, int ldr, int a, double *Ri) {
    for (int j = threadIdx.x + blockIdx.x * blockDim.x; j < a; j += blockDim.x * gridDim.x) {
        for (int i = a - 1; i >= 0; --i) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int k = i + 1; k <= j; ++k) s -= R[i + (long long)k * ldr] * Ri[k + (long long)j * a];
            Ri[i + (long long)j * a] = (i <= j) ? s / R[i + (long long)i * ldr] : 0.0;
        }
    }
}

// Per lane: G (k x k, stored in gw) -> G^-1 (in place) via Cholesky.
__global__ void __launch_bounds__(128) k_lane_inv(double *gw, const int *kdef, int *info) {
    const int l = blockIdx.x;
    const int k = kdef[l];
    double *G = gw + (long long)l * KMAX * KMAX;
    __shared__ double L[KMAX * KMAX];
    __shared__ double Li[KMAX * KMAX];
    __shared__ int fail;
    if (threadIdx.x == 0) fail = 0;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int i = e % k, j = e / k;
        // symmetrise: use the mean of the two triangles
        L[i + j * KMAX] = 0.5 * (G[i + j * KMAX] + G[j + i * KMAX]);
    }
    __syncthreads();
    for (int c = 0; c < k; ++c) {
        if (threadIdx.x == 0) {
            const double d = L[c + c * KMAX];
            if (bad(d)) fail = c + 1;
            else L[c + c * KMAX] = sqrt(d);
        }
        __syncthreads();
        if (fail) break;
        for (int i = c + 1 + threadIdx.x; i < k; i += blockDim.x) L[i + c * KMAX] /= L[c + c * KMAX];
        __syncthreads();
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            const int i = e % k, j = e / k;
            if (i > c && j > c && i >= j) L[i + j * KMAX] -= L[i + c * KMAX] * L[j + c * KMAX];
        }
        __syncthreads();
    }
    if (fail) {
        if (threadIdx.x == 0 && info) atomicMax(info, 1);
        return;
    }
    // Li = L^-1 (column j by forward substitution)
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        for (int i = 0; i < k; ++i) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int q = j; q < i; ++q) s -= L[i + q * KMAX] * Li[q + j * KMAX];
            Li[i + j * KMAX] = (i >= j) ? s / L[i + i * KMAX] : 0.0;
        }
    }
    __syncthreads();
    // G^-1 = Li^T Li
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int i = e % k, j = e / k;
        const int q0 = i > j ? i : j;
        double s = 0.0;
        for (int q = q0; q < k; ++q) s += Li[q + i * KMAX] * Li[q + j * KMAX];
        G[i + j * KMAX] = s;
    }
}

// Cyclic Jacobi eigen-decomposition of a symmetric k x k matrix (one thread;
// k is small).  A is overwritten; eigenvalues ascending with vectors.
__global__ void k_jacobi(double *A, int lda, int k, double *Q, double *w) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Q[i + (long long)j * k] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                const double v = A[i + (long long)j * lda];
                tot += v * v;
                if (i != j) off += v * v;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = A[p + (long long)q * lda];
                if (apq == 0.0) continue;
                const double app = A[p + (long long)p * lda], aqq = A[q + (long long)q * lda];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < k; ++r) {
                    const double arp = A[r + (long long)p * lda], arq = A[r + (long long)q * lda];
                    A[r + (long long)p * lda] = c * arp - s * arq;
                    A[r + (long long)q * lda] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {
                    const double apr = A[p + (long long)r * lda], aqr = A[q + (long long)r * lda];
                    A[p + (long long)r * lda] = c * apr - s * aqr;
                    A[q + (long long)r * lda] = s * apr + c * aqr;
                }
                for (int r = 0; r < k; ++r) {
                    const double qrp = Q[r + (long long)p * k], qrq = Q[r + (long long)q * k];
                    Q[r + (long long)p * k] = c * qrp - s * qrq;
                    Q[r + (long long)q * k] = s * qrp + c * qrq;
                }
            }
    }
    // sort ascending (selection sort, swapping vectors)
    for (int i = 0; i < k; ++i) w[i] = A[i + (long long)i * lda];
    for (int i = 0; i < k; ++i) {
        int mi = i;
        for (int j = i + 1; j < k; ++j)
            if (w[j] < w[mi]) mi = j;
        if (mi != i) {
            const double t = w[i]; w[i] = w[mi]; w[mi] = t;
            for (int r = 0; r < k; ++r) {
                const double a = Q[r + (long long)i * k];
                Q[r + (long long)i * k] = Q[r + (long long)mi * k];
                Q[r + (long long)mi * k] = a;
            }
        }
    }
}

// ---------------------------------------------------------------- parallel Jacobi
// Cyclic Jacobi for a symmetric m2 x m2 matrix (m2 even), all disjoint pairs of
// a round at once (round-robin / circle ordering): round t pairs index t with
// m2 - 1 and (t + k) mod (m2 - 1) with (t - k) mod (m2 - 1), k = 1 .. m2/2 - 1;
// the m2 - 1 rounds of a sweep meet every pair once.  Each pair's rotation is
// the symmetric 2 x 2 Schur rotation of Golub and Van Loan (Matrix
// Computations, Sec. 8.5: "sym.schur2"), which zeroes A(p, q).
__device__ __forceinline__ void jac_pair(int m2, int t, int k, int &p, int &q) {
    const int half = m2 - 1;
    int i, j;
    if (k == 0) { i = t; j = m2 - 1; }
    else { i = (t + k) % half; j = (t - k + half) % half; }
    p = i < j ? i : j;
    q = i < j ? j : i;
}

__global__ void k_jac_params(const double *__restrict__ A, int lda, int m2, int t, double *__restrict__ cs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m2 / 2) return;
    int p, q;
    jac_pair(m2, t, k, p, q);
    const double apq = A[p + (long long)q * lda];
    double c = 1.0, sn = 0.0;
    if (apq != 0.0) {
        const double tau = (A[q + (long long)q * lda] - A[p + (long long)p * lda]) / (2.0 * apq);
        const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        c = 1.0 / sqrt(1.0 + tt * tt);
        sn = tt * c;
    }
    cs[2 * k] = c;
    cs[2 * k + 1] = sn;
}

// A <- J^T A J and Q <- Q J for the round's rotations J (block-diagonal in the
// pairs): one thread per 2 x 2 block (pair a, pair b) of A, read and written in
// place, then one per (row of Q, pair).
__global__ void k_jac_apply(double *__restrict__ A, int lda, int m2, int t, const double *__restrict__ cs,
                            double *__restrict__ Q, int ldq) {
    const int np = m2 / 2;
    const long long nb = (long long)np * np, tot = nb + (long long)m2 * np;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < nb) {
            const int a = (int)(e % np), b = (int)(e / np);
            int pa, qa, pb, qb;
            jac_pair(m2, t, a, pa, qa);
            jac_pair(m2, t, b, pb, qb);
            const double ca = cs[2 * a], sa = cs[2 * a + 1], cb = cs[2 * b], sb = cs[2 * b + 1];
            double *a11 = A + pa + (long long)pb * lda, *a12 = A + pa + (long long)qb * lda;
            double *a21 = A + qa + (long long)pb * lda, *a22 = A + qa + (long long)qb * lda;
            const double t11 = ca * *a11 - sa * *a21, t12 = ca * *a12 - sa * *a22;   // J_a^T A_ab
            const double t21 = sa * *a11 + ca * *a21, t22 = sa * *a12 + ca * *a22;
            *a11 = t11 * cb - t12 * sb;                                              // ... J_b
            *a12 = t11 * sb + t12 * cb;
            *a21 = t21 * cb - t22 * sb;
            *a22 = t21 * sb + t22 * cb;
        } else {
            const long long f = e - nb;
            const int row = (int)(f % m2), b = (int)(f / m2);
            int pb, qb;
            jac_pair(m2, t, b, pb, qb);
            const double cb = cs[2 * b], sb = cs[2 * b + 1];
            double *qp = Q + row + (long long)pb * ldq, *qq = Q + row + (long long)qb * ldq;
            const double x = *qp, y = *qq;
            *qp = x * cb - y * sb;
            *qq = x * sb + y * cb;
        }
    }
}

// out[0] += sum of squares off the diagonal, out[1] += all squares.
__global__ void k_jac_offnorm(const double *__restrict__ A, int lda, int m2, double *__restrict__ out) {
    double off = 0.0, all = 0.0;
    const long long tot = (long long)m2 * m2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % m2), j = (int)(e / m2);
        const double v = A[i + (long long)j * lda];
        all += v * v;
        if (i != j) off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_down_sync(0xffffffffu, off, o);
        all += __shfl_down_sync(0xffffffffu, all, o);
    }
    if ((threadIdx.x & 31) == 0) { atomicAdd(out, off); atomicAdd(out + 1, all); }
}

__global__ void k_eye(double *__restrict__ Q, int ldq, int m2) {
    const long long tot = (long long)m2 * m2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x)
        Q[(e % m2) + (e / m2) * (long long)ldq] = (e % m2 == e / m2) ? 1.0 : 0.0;
}

}  // namespace

// Shared-memory attribute for the staged kernels (per device ordinal).
void sm_attr(const void *f, int bytes) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void *, int>, int>> done;   // (func, dev) -> bytes set
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    for (auto &e : done)
        if (e.first.first == f && e.first.second == dev) {
            if (e.second >= bytes) return;
            RCG_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
            e.second = bytes;
            return;
        }
    RCG_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done.push_back({{f, dev}, bytes});
}

void chol_run(cudaStream_t st, double *A, int lda, long long strideA, int k0, int r, int *info, int nbatch) {
    if (r <= SM_R) {
        const int bytes = (int)(sizeof(double) * (size_t)r * r);
        if (bytes > 48 * 1024) sm_attr((const void *)k_chol_sm, bytes);
        k_chol_sm<<<nbatch, 1024, bytes, st>>>(A, lda, strideA, k0, r, info);
        count_launch();
        RCG_CHECK_LAUNCH();
        return;
    }
    for (int b = 0; b < nbatch; ++b) {
        k_chol<<<1, 1024, 0, st>>>(A + b * strideA, lda, k0, r, info);
        count_launch();
        RCG_CHECK_LAUNCH();
    }
}

// Eigen-decomposition of the symmetric m2 x m2 matrix A (m2 even; ld lda):
// on return diag(A) holds the eigenvalues and Q (ld ldq) the eigenvectors.
// Sweeps until the off-diagonal mass is below tol^2 of the total (at most
// max_sweeps); cs: m2 doubles, red: 2 doubles of device scratch.  Returns the
// number of sweeps (host synchronisation once per sweep).
int jacobi_parallel(cudaStream_t st, double *A, int lda, int m2, double *Q, int ldq, double *cs, double *red,
                    double tol, int max_sweeps) {
    if (m2 <= 0) return 0;
    if (m2 & 1) throw Error{RCG_ERR_INVALID, "jacobi_parallel: odd order"};
    const long long work = (long long)(m2 / 2) * (m2 / 2) + (long long)m2 * (m2 / 2);
    const int blocks = (int)std::min<long long>((work + 255) / 256, 4 * 152);
    const unsigned gsq = (unsigned)std::min<long long>(((long long)m2 * m2 + 255) / 256, 1024);
    k_eye<<<gsq, 256, 0, st>>>(Q, ldq, m2);
    count_launch();
    RCG_CHECK_LAUNCH();
    double h[2];
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        RCG_CUDA_TRY(cudaMemsetAsync(red, 0, 2 * sizeof(double), st));
        k_jac_offnorm<<<gsq, 256, 0, st>>>(A, lda, m2, red);
        count_launch();
        RCG_CHECK_LAUNCH();
        RCG_CUDA_TRY(cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, st));
        RCG_CUDA_TRY(cudaStreamSynchronize(st));
        if (!(h[0] > tol * tol * h[1])) break;
        for (int t = 0; t < m2 - 1; ++t) {
            k_jac_params<<<(m2 / 2 + 127) / 128, 128, 0, st>>>(A, lda, m2, t, cs);
            k_jac_apply<<<blocks, 256, 0, st>>>(A, lda, m2, t, cs, Q, ldq);
            count_launch();
            count_launch();
        }
        RCG_CHECK_LAUNCH();
    }
    return sweep;
}

void chol_inplace(cudaStream_t st, double *A, int lda, int r, int *info) {
    if (r <= 0) return;
    chol_run(st, A, lda, 0, 0, r, info, 1);
}

void chol_batched(cudaStream_t st, double *A, int lda, long long strideA, int r, int nbatch, int *info) {
    if (r <= 0 || nbatch <= 0) return;
    chol_run(st, A, lda, strideA, 0, r, info, nbatch);
}

void chol_border(cudaStream_t st, double *L, int ldl, int r_old, int a, int *info) {
    if (a <= 0) return;
    if (r_old > 0) {
        k_chol_border<<<1, 1024, 0, st>>>(L, ldl, r_old, a);
        count_launch();
        RCG_CHECK_LAUNCH();
    }
    chol_run(st, L, ldl, 0, r_old, r_old + a, info, 1);
}

void trsv_multi(cudaStream_t st, const double *L, int ldl, long long strideL, int r, double *B, int ldb,
                long long strideB, int m, int nbatch, bool transpose) {
    if (r <= 0 || m <= 0 || nbatch <= 0) return;
    if (r <= SM_R) {
        const int bytes = (int)(sizeof(double) * ((size_t)r * r + r + 8 * (size_t)r));
        if (bytes > 48 * 1024) sm_attr((const void *)k_trsv_sm, bytes);
        k_trsv_sm<<<dim3((m + 7) / 8, nbatch), 256, bytes, st>>>(L, ldl, strideL, r, B, ldb, strideB, m,
                                                                transpose ? 1 : 0);
        count_launch();
        RCG_CHECK_LAUNCH();
        return;
    }
    for (int b = 0; b < nbatch; ++b) trsv_lower_batched(st, L + b * strideL, ldl, r, B + b * strideB, ldb, m, transpose);
}

void trsv_lower_batched(cudaStream_t st, const double *L, int ldl, int r, double *B, int ldb, int m,
                        bool transpose) {
    if (r <= 0 || m <= 0) return;
    if (r <= SM_R) {
        trsv_multi(st, L, ldl, 0, r, B, ldb, 0, m, 1, transpose);
        return;
    }
    const size_t sh = sizeof(double) * (size_t)r;
    if (sh > 48 * 1024)
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_trsv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    k_trsv<<<m, 256, sh, st>>>(L, ldl, r, B, ldb, transpose ? 1 : 0);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void ordered_drop_chol(cudaStream_t st, const double *M, int a, const double *xnorm2, double *S, double tau,
                       double *R, int *kept, double *ratio) {
    if (a <= 0) return;
    const size_t sm = sizeof(double) * (size_t)a;
    if (sm > 48 * 1024) RCG_CUDA_TRY(cudaFuncSetAttribute(k_ordered_drop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_ordered_drop<<<1, 1024, sm, st>>>(M, a, xnorm2, tau, S, R, kept, ratio);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void tri_upper_inverse(cudaStream_t st, const double *R, int ldr, int a, double *Ri) {
    if (a <= 0) return;
    k_tri_upper_inv<<<(a + 127) / 128, 128, 0, st>>>(R, ldr, a, Ri);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void lane_inverse(cudaStream_t st, double *gw, const int *kdef, int m, int *info) {
    if (m <= 0) return;
    k_lane_inv<<<m, 128, 0, st>>>(gw, kdef, info);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void jacobi_eig(cudaStream_t st, double *A, int lda, int k, double *Q, double *w) {
    k_jacobi<<<1, 32, 0, st>>>(A, lda, k, Q, w);
    count_launch();
    RCG_CHECK_LAUNCH();
}

}  // namespace rcg
