// Diffusion tracking the absorption: D(x; p) = 1 / (3 (mu(x; p) + mu_s'))
// at every parameter point (an extension of Sec. 2.1, where D is fixed).
//
// A~(p) then changes off the diagonal as well (every face weight of eq. H's
// stencil and the Robin term D_p / (1 + alpha_p) of the elimination in Sec. 3),
// and so do the effective source and detector weights of Sec. 3.1.  The
// kernels here build, per sample or parameter point,
//   * D, the face weights W (towards +x, +y, +z) and the diagonal
//     (k_d_of_mu, then the fixed-D set-up kernels on that D);
//   * the difference or derivative of A~ as a diagonal dg and face weights
//     dw (k_track_deriv: dD = -3 D^2 dmu, Robin face dD / (1 + alpha)^2);
//   * the rows where such a difference is not zero (k_touch, then the block
//     list of the tensor-core weighted products);
//   * on those rows, Y = dA X in float64 next to the rows of X (k_delta_rows),
//     so that V^T dA V is a product over few rows (Galerkin matrices of the
//     check, the reduced matrix and the Jacobian of eq. newjac);
//   * the source / detector weights at a D and their derivatives
//     (k_rhs_weights), and the Jacobian's terms from them (k_jac_rhs).
#include "common.cuh"

#include <algorithm>

namespace rcg {
namespace {

int grid1(long long n) { return (int)std::max(1LL, std::min((n + 255) / 256, 4096LL)); }

__global__ void k_d_of_mu(long long n, const double *__restrict__ mu, double mus, double *__restrict__ D64,
                          float *__restrict__ D32) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const double d = 1.0 / (3.0 * (mu[p] + mus));
        D64[p] = d;
        if (D32) D32[p] = (float)d;
    }
}

// dg = scale (sum over p's faces of dw_f + h^2 dmu_p), dw (+x, +y, +z faces)
// = scale dw_f with dD = -3 D^2 dmu: interior face (dD_p + dD_q)/2, ghost face
// dD_p, Robin face dD_p / (1 + alpha_p)^2.
__global__ void k_track_deriv(Grid g, const double *__restrict__ D, const double *__restrict__ dmu, double h,
                              double robin_A, double scale, double *__restrict__ dg, double *__restrict__ dw) {
    const long long sxy = (long long)g.Nx * g.Ny;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.Nx);
        const long long rest = p / g.Nx;
        const int j = (int)(rest % g.Ny), k = (int)(rest / g.Ny);
        auto dD = [&](long long q) { return -3.0 * D[q] * D[q] * dmu[q]; };
        const double dp = dD(p);
        const double wxp = i < g.Nx - 1 ? 0.5 * (dp + dD(p + 1)) : 0.0;
        const double wyp = (g.Ny > 1 && j < g.Ny - 1) ? 0.5 * (dp + dD(p + g.Nx)) : 0.0;
        const double wzp = k < g.Nz - 1 ? 0.5 * (dp + dD(p + sxy)) : 0.0;
        const double alpha = 2.0 * robin_A * D[p] / h;
        const double robin = dp / ((1.0 + alpha) * (1.0 + alpha));
        double s = h * h * dmu[p];
        s += i > 0 ? 0.5 * (dp + dD(p - 1)) : dp;
        s += i < g.Nx - 1 ? wxp : dp;
        if (g.Ny > 1) {
            s += j > 0 ? 0.5 * (dp + dD(p - g.Nx)) : dp;
            s += j < g.Ny - 1 ? wyp : dp;
        }
        s += k > 0 ? 0.5 * (dp + dD(p - sxy)) : robin;
        s += k < g.Nz - 1 ? wzp : robin;
        dg[p] = scale * s;
        dw[p] = scale * wxp;
        dw[g.ld + p] = scale * wyp;
        dw[2 * g.ld + p] = scale * wzp;
    }
}

// touch[p] = |dg_p| + |dw| of the six faces of p: nonzero exactly on the rows of dA
__global__ void k_touch(Grid g, const double *__restrict__ dg, const double *__restrict__ dw, double *__restrict__ touch) {
    const long long sxy = (long long)g.Nx * g.Ny;
    const double *wx = dw, *wy = dw + g.ld, *wz = dw + 2 * g.ld;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.Nx);
        const long long rest = p / g.Nx;
        const int j = (int)(rest % g.Ny), k = (int)(rest / g.Ny);
        double t = fabs(dg[p]) + fabs(wx[p]) + fabs(wy[p]) + fabs(wz[p]);
        if (i > 0) t += fabs(wx[p - 1]);
        if (j > 0) t += fabs(wy[p - g.Nx]);
        if (k > 0) t += fabs(wz[p - sxy]);
        touch[p] = t;
    }
}

// For the rows of listed 32-row blocks b0 .. b0 + nb - 1 and column c =
// blockIdx.y: Xc = x_p, Yc = dg_p x_p - sum over faces dw_f x_q (float64).
// Rows past n are written as zeros.  Compact layout: row (b - b0) 32 + lane, ld ldc.
template <typename T>
__global__ void __launch_bounds__(256)
k_delta_rows(Grid g, const int *__restrict__ blist, int b0, int nb, const double *__restrict__ dg,
             const double *__restrict__ dw, const T *__restrict__ X, long long ldx, T *__restrict__ Xc,
             double *__restrict__ Yc, long long ldc) {
    const int bl = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (bl >= nb) return;
    const int c = blockIdx.y;
    const long long p = (long long)blist[b0 + bl] * 32 + (threadIdx.x & 31);
    const long long row = (long long)bl * 32 + (threadIdx.x & 31);
    const T *x = X + (long long)c * ldx;
    double xv = 0.0, y = 0.0;
    if (p < g.n) {
        const long long sxy = (long long)g.Nx * g.Ny;
        const int i = (int)(p % g.Nx);
        const long long rest = p / g.Nx;
        const int j = (int)(rest % g.Ny), k = (int)(rest / g.Ny);
        const double *wx = dw, *wy = dw + g.ld, *wz = dw + 2 * g.ld;
        xv = (double)x[p];
        y = dg[p] * xv;
        if (i > 0) y -= wx[p - 1] * (double)x[p - 1];
        if (i < g.Nx - 1) y -= wx[p] * (double)x[p + 1];
        if (j > 0) y -= wy[p - g.Nx] * (double)x[p - g.Nx];
        if (j < g.Ny - 1) y -= wy[p] * (double)x[p + g.Nx];
        if (k > 0) y -= wz[p - sxy] * (double)x[p - sxy];
        if (k < g.Nz - 1) y -= wz[p] * (double)x[p + sxy];
    }
    Xc[(long long)c * ldc + row] = (T)xv;
    Yc[(long long)c * ldc + row] = y;
}

// Effective weights at D (Sec. 3.1): source j < nsrc: s_j D_p / (1 + alpha_p),
// detector: c_j alpha_p / (1 + alpha_p), alpha_p = 2 A D_p / h at its node p.
// With dmu (nparam columns of stride lddmu): dwt[k nrhs + j] = the derivative in
// p_k through D (dD = -3 D^2 dmu): s_j dD / (1 + alpha)^2, c_j (2A/h) dD / (1 + alpha)^2.
__global__ void k_rhs_weights(const double *__restrict__ D, const int *__restrict__ node, const double *__restrict__ wt,
                              int nsrc, int nrhs, double robin_A, double h, double *__restrict__ w,
                              const double *__restrict__ dmu, long long lddmu, int nparam, double *__restrict__ dwt) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nrhs) return;
    const long long p = node[j];
    const double Dp = D[p], alpha = 2.0 * robin_A * Dp / h;
    const bool src = j < nsrc;
    if (w) w[j] = wt[j] * (src ? Dp / (1.0 + alpha) : alpha / (1.0 + alpha));
    if (dmu) {
        const double dfac = wt[j] * (src ? 1.0 : 2.0 * robin_A / h) / ((1.0 + alpha) * (1.0 + alpha));
        for (int k = 0; k < nparam; ++k)
            dwt[(long long)k * nrhs + j] = dfac * (-3.0 * Dp * Dp * dmu[(long long)k * lddmu + p]);
    }
}

// J_k[d, s] += dwt_k[nsrc + d] Pd[d, s] + dwt_k[s] Ps[s, d]  (Pd = (V X_r) at the
// detector nodes, nd x ns; Ps = (V Z_r) at the source nodes, ns x nd)
__global__ void k_jac_rhs(int nparam, int nd, int ns, const double *__restrict__ dwt, const double *__restrict__ Pd,
                          const double *__restrict__ Ps, double *__restrict__ J) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per = (long long)nd * ns;
    if (e >= per * nparam) return;
    const int k = (int)(e / per);
    const int rem = (int)(e % per), d = rem % nd, s = rem / nd;
    const double *dw = dwt + (long long)k * (nd + ns);
    J[e] += dw[ns + d] * Pd[d + (long long)nd * s] + dw[s] * Ps[s + (long long)ns * d];
}

// dst_c = beta_c x_c (n elements) with beta_c = w1[c] / w0[c]
__global__ void k_ratio_scale(long long n, const double *__restrict__ x, long long ldx, const double *__restrict__ w1,
                              const double *__restrict__ w0, double *__restrict__ dst, long long ldd) {
    const int c = blockIdx.y;
    const double b = w1[c] / w0[c];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        dst[(long long)c * ldd + p] = b * x[(long long)c * ldx + p];
}

}  // namespace

void track_coefficients(cudaStream_t st, const Grid &g, const double *mu, double mus, double h, double robin_A,
                        double *D64, float *D32, double *W64, double *diag64, float *diag32) {
    Grid g0 = g;
    g0.Ds64 = nullptr; g0.Ws64 = nullptr; g0.Ds32 = nullptr;
    k_d_of_mu<<<grid1(g.n), 256, 0, st>>>(g.n, mu, mus, D64, D32);
    count_launch();
    RCG_CHECK_LAUNCH();
    face_weights(st, g0, D64, W64);
    diag_star(st, g0, D64, h, robin_A, diag64);
    diag_sample(st, g.n, diag64, mu, h * h, diag64, diag32);
}

void track_deriv(cudaStream_t st, const Grid &g, const double *D, const double *dmu, double h, double robin_A,
                 double scale, double *dg, double *dw) {
    k_track_deriv<<<grid1(g.n), 256, 0, st>>>(g, D, dmu, h, robin_A, scale, dg, dw);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void track_touch(cudaStream_t st, const Grid &g, const double *dg, const double *dw, double *touch) {
    k_touch<<<grid1(g.n), 256, 0, st>>>(g, dg, dw, touch);
    count_launch();
    RCG_CHECK_LAUNCH();
}

template <typename T>
void delta_rows(cudaStream_t st, const Grid &g, const int *blist, int b0, int nb, const double *dg, const double *dw,
                const T *X, long long ldx, int ncols, T *Xc, double *Yc, long long ldc) {
    if (nb <= 0 || ncols <= 0) return;
    if (ncols > 65535) throw Error{RCG_ERR_INVALID, "delta_rows: too many columns"};
    k_delta_rows<T><<<dim3((unsigned)((nb + 7) / 8), (unsigned)ncols), 256, 0, st>>>(g, blist, b0, nb, dg, dw, X, ldx,
                                                                                    Xc, Yc, ldc);
    count_launch();
    RCG_CHECK_LAUNCH();
}
template void delta_rows<float>(cudaStream_t, const Grid &, const int *, int, int, const double *, const double *,
                                const float *, long long, int, float *, double *, long long);
template void delta_rows<double>(cudaStream_t, const Grid &, const int *, int, int, const double *, const double *,
                                 const double *, long long, int, double *, double *, long long);

void rhs_weights(cudaStream_t st, const double *D, const int *node, const double *wt, int nsrc, int nrhs,
                 double robin_A, double h, double *w, const double *dmu, long long lddmu, int nparam, double *dwt) {
    if (nrhs <= 0) return;
    k_rhs_weights<<<(nrhs + 127) / 128, 128, 0, st>>>(D, node, wt, nsrc, nrhs, robin_A, h, w, dmu, lddmu, nparam, dwt);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void jac_rhs_terms(cudaStream_t st, int nparam, int nd, int ns, const double *dwt, const double *Pd, const double *Ps,
                   double *J) {
    const long long tot = (long long)nparam * nd * ns;
    if (tot <= 0) return;
    k_jac_rhs<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nparam, nd, ns, dwt, Pd, Ps, J);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void ratio_scale(cudaStream_t st, long long n, const double *x, long long ldx, const double *w1, const double *w0,
                 double *dst, long long ldd, int ncols) {
    if (ncols <= 0) return;
    k_ratio_scale<<<dim3(grid1(n), (unsigned)ncols), 256, 0, st>>>(n, x, ldx, w1, w0, dst, ldd);
    count_launch();
    RCG_CHECK_LAUNCH();
}

}  // namespace rcg
