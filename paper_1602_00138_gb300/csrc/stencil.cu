// Matrix-free application of the Schur-complement diffusion operator
// A~_s = A~_* + diag(h^2 mu_s) (Sec. 3, eq. sum) on batches of columns.
//
//   (A~ x)_p = diag_s[p] x_p - sum_{interior neighbours q} w_pq x_q,
//   w_pq = (D_p + D_q) / 2,
//   diag_s[p] = sum_faces w_f^eff + h^2 mu_s[p]   (precomputed, see api.cu)
//
// The lateral Dirichlet ghosts and the eliminated Robin unknowns only touch
// the diagonal, so the off-diagonal part is a plain 5/7-point stencil on the
// unknown grid.  Face weights are formed on the fly from D (one coefficient
// stream, the neighbours come from L1/L2), amortised over the NB columns a
// thread handles.
#include "common.cuh"

#include <algorithm>

namespace rcg {

thread_local long long *g_launch_counter = nullptr;
thread_local long long g_spin_budget = 0;

namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ T half_sum(T a, T b) { return T(0.5) * (a + b); }

template <int NB>
__device__ __forceinline__ void block_reduce_add(double (&acc)[NB], double *out, const bool (&act)[NB]) {
    __shared__ double red[kThreads / 32][NB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        double v = acc[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][t] = v;
    }
    __syncthreads();
    if (threadIdx.x < NB) {
        const int t = threadIdx.x;
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w][t];
        if (act[t]) atomicAdd(out + t, s);
    }
}

// y_c = A~_{s(c)} x_c for column c = blockIdx.y; optional dot x_c^T y_c.
// One column per CTA row and one node per thread keep the register count low
// so that enough warps are resident to cover the HBM latency; the column's
// pointers are uniform per CTA (no per-node pointer loads).  The neighbour
// values come from L1/L2 (x +- 1 from the same warp's lines).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_apply(Grid g, const T *__restrict__ D, const T *const *__restrict__ diag_of_col,
        const T *const *__restrict__ src, T *const *__restrict__ dst, int ncols,
        const int *__restrict__ active, double *__restrict__ dots, unsigned long long *__restrict__ act_count) {
    const int c = blockIdx.y;
    if (c >= ncols || (active != nullptr && active[c] == 0)) return;
    if (act_count && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(act_count, 1ULL);
    const T *__restrict__ x = src[c];
    T *__restrict__ y = dst[c];
    const T *__restrict__ dg = diag_of_col[c];
    D = sample_D(g, dg, D);
    const int sxy = g.Nx * g.Ny;          // grids here are < 2^31 nodes (checked at rcg_create)
    const int nn = (int)g.n;
    const bool has_y = g.Ny > 1;
    T acc = T(0);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += gridDim.x * blockDim.x) {
        const int i = p % g.Nx;
        const int rest = p / g.Nx;
        const int j = rest % g.Ny;
        const int k = rest / g.Ny;
        const T Dp = D[p];
        const T xc = x[p];
        T v = dg[p] * xc;
        if (i > 0) v -= half_sum(Dp, D[p - 1]) * x[p - 1];
        if (i < g.Nx - 1) v -= half_sum(Dp, D[p + 1]) * x[p + 1];
        if (has_y && j > 0) v -= half_sum(Dp, D[p - g.Nx]) * x[p - g.Nx];
        if (has_y && j < g.Ny - 1) v -= half_sum(Dp, D[p + g.Nx]) * x[p + g.Nx];
        if (k > 0) v -= half_sum(Dp, D[p - sxy]) * x[p - sxy];
        if (k < g.Nz - 1) v -= half_sum(Dp, D[p + sxy]) * x[p + sxy];
        y[p] = v;
        acc += xc * v;
    }
    if (dots) {
        double v = (double)acc;
        __shared__ double red[kThreads / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s2 = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s2 += red[w];
            atomicAdd(dots + c, s2);
        }
    }
}

// r_c = b_c - A~_{s(c)} x_c in float64, b_c = bw_c e_{node_c}; optional float32 copy; rr_c += r^T r.
// TRACK: every column reads the face weights of its own sample (diffusion
// tracking the absorption); otherwise W is shared and read once per node.
template <int NB, bool TRACK>
__global__ void __launch_bounds__(kThreads)
k_residual64(Grid g, const double *__restrict__ W, const double *const *__restrict__ diag_of_col,
             const double *const *__restrict__ xsrc, double *const *__restrict__ rdst,
             float *const *__restrict__ r32dst, int ncols, const int *__restrict__ node,
             const double *__restrict__ bw, double *__restrict__ rr, const int *__restrict__ active) {
    // W: face weights (D_p + D_q)/2 towards the +x, +y, +z neighbour (0 on the
    // last layer of each axis), three columns of stride g.ld
    const int c0 = blockIdx.y * NB;
    bool act[NB];
    bool any = false;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        const int c = c0 + t;
        act[t] = (c < ncols) && (active == nullptr || active[c] != 0);
        any |= act[t];
    }
    if (!any) return;
    double acc[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) acc[t] = 0.0;
    const int sxy = g.Nx * g.Ny, n = (int)g.n;
    const double *__restrict__ Wx = W, *__restrict__ Wy = W + g.ld, *__restrict__ Wz = W + 2 * g.ld;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int i = p % g.Nx, rest = p / g.Nx;
        const int j = rest % g.Ny, k = rest / g.Ny;
        double wxm = 0.0, wxp = 0.0, wym = 0.0, wyp = 0.0, wzm = 0.0, wzp = 0.0;
        if constexpr (!TRACK) {
            wxm = i > 0 ? Wx[p - 1] : 0.0; wxp = Wx[p];
            wym = j > 0 ? Wy[p - g.Nx] : 0.0; wyp = Wy[p];
            wzm = k > 0 ? Wz[p - sxy] : 0.0; wzp = Wz[p];
        }
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            if (!act[t]) continue;
            const int c = c0 + t;
            const double *x = xsrc[c];
            const double *dgc = diag_of_col[c];
            double v = dgc[p] * x[p];
            if constexpr (TRACK) {
                const double *Wc = sample_W(g, dgc, W);
                const double *Wcx = Wc, *Wcy = Wc + g.ld, *Wcz = Wc + 2 * g.ld;
                if (i > 0) v -= Wcx[p - 1] * x[p - 1];
                if (i < g.Nx - 1) v -= Wcx[p] * x[p + 1];
                if (j > 0) v -= Wcy[p - g.Nx] * x[p - g.Nx];
                if (j < g.Ny - 1) v -= Wcy[p] * x[p + g.Nx];
                if (k > 0) v -= Wcz[p - sxy] * x[p - sxy];
                if (k < g.Nz - 1) v -= Wcz[p] * x[p + sxy];
            } else {
                if (i > 0) v -= wxm * x[p - 1];
                if (i < g.Nx - 1) v -= wxp * x[p + 1];
                if (j > 0) v -= wym * x[p - g.Nx];
                if (j < g.Ny - 1) v -= wyp * x[p + g.Nx];
                if (k > 0) v -= wzm * x[p - sxy];
                if (k < g.Nz - 1) v -= wzp * x[p + sxy];
            }
            const double b = (p == node[c]) ? bw[c] : 0.0;
            const double res = b - v;
            if (rdst) rdst[c][p] = res;
            if (r32dst) r32dst[c][p] = (float)res;
            acc[t] += res * res;
        }
    }
    if (rr) block_reduce_add<NB>(acc, rr + c0, act);
}

// W[a * ld + p] = (D_p + D_q) / 2 with q the +a neighbour of p (0 if p is on
// the last layer of axis a): the off-diagonal couplings of A~ (Sec. 3).
__global__ void k_face_weights(Grid g, const double *__restrict__ D, double *__restrict__ W) {
    const int sxy = g.Nx * g.Ny;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.n; p += (long long)gridDim.x * blockDim.x) {
        const int pi = (int)p;
        const int i = pi % g.Nx, rest = pi / g.Nx, j = rest % g.Ny, k = rest / g.Ny;
        W[p] = i < g.Nx - 1 ? 0.5 * (D[p] + D[p + 1]) : 0.0;
        W[g.ld + p] = j < g.Ny - 1 ? 0.5 * (D[p] + D[p + g.Nx]) : 0.0;
        W[2 * g.ld + p] = k < g.Nz - 1 ? 0.5 * (D[p] + D[p + sxy]) : 0.0;
    }
}

int grid_x_for(long long n, int groups) {
    // about 4 resident CTAs per SM over all groups, at least one node per thread
    int sms = 152;
    static int cached = 0;
    if (!cached) {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) {
            int v = 0;
            if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
                cached = v;
        }
        if (!cached) cached = 152;
    }
    sms = cached;
    long long want = (4LL * sms + groups - 1) / groups;
    long long maxb = (n + kThreads - 1) / kThreads;
    long long gx = want < maxb ? want : maxb;
    if (gx < 1) gx = 1;
    return (int)gx;
}

}  // namespace

template <typename T>
void apply_op(cudaStream_t st, const Grid &g, const T *D, const T *const *diag_of_col,
              const T *const *src, T *const *dst, int ncols, const int *active,
              double *dots, unsigned long long *act_count) {
    if (ncols <= 0) return;
    // ~8 resident CTAs per SM over all columns, at least one node per thread
    long long want = (8LL * 152 + ncols - 1) / ncols;
    long long maxb = (g.n + kThreads - 1) / kThreads;
    const int gx = (int)std::max(1LL, std::min(want, maxb));
    dim3 grid(gx, ncols);
    k_apply<T><<<grid, kThreads, 0, st>>>(g, D, diag_of_col, src, dst, ncols, active, dots, act_count);
    count_launch();
    RCG_CHECK_LAUNCH();
}

template void apply_op<double>(cudaStream_t, const Grid &, const double *, const double *const *,
                               const double *const *, double *const *, int, const int *, double *,
                               unsigned long long *);
template void apply_op<float>(cudaStream_t, const Grid &, const float *, const float *const *,
                              const float *const *, float *const *, int, const int *, double *,
                              unsigned long long *);

void residual64(cudaStream_t st, const Grid &g, const double *W, const double *const *diag_of_col,
                const double *const *x, double *const *r, float *const *r32, int ncols,
                const int *node, const double *bw, double *rr, const int *active, int nact) {
    if (ncols <= 0) return;
    constexpr int NB = 8;
    const int groups = (ncols + NB - 1) / NB;
    // CTAs per group for the groups that hold selected columns (at most nact of
    // them; the others exit at once): a restart of a few lanes keeps the GPU busy
    const int busy = std::max(1, std::min(groups, nact < 0 ? ncols : nact));
    dim3 grid(grid_x_for(g.n, busy), groups);
    if (g.Ws64)
        k_residual64<NB, true><<<grid, kThreads, 0, st>>>(g, W, diag_of_col, x, r, r32, ncols, node, bw, rr, active);
    else
        k_residual64<NB, false><<<grid, kThreads, 0, st>>>(g, W, diag_of_col, x, r, r32, ncols, node, bw, rr, active);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void face_weights(cudaStream_t st, const Grid &g, const double *D, double *W) {
    k_face_weights<<<(unsigned)std::min<long long>((g.n + 255) / 256, 4096), 256, 0, st>>>(g, D, W);
    count_launch();
    RCG_CHECK_LAUNCH();
}

}  // namespace rcg
