// Internal declarations of librcg: device buffers, launch helpers and the
// kernels' host-side launchers.  See include/rcg.h for the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/rcg.h"

namespace rcg {

// ---------------------------------------------------------------- errors
struct Error {
    int code;
    std::string msg;
};

#define RCG_STR2(x) #x
#define RCG_STR(x) RCG_STR2(x)
#define RCG_WHERE " (" __FILE__ ":" RCG_STR(__LINE__) ")"

#define RCG_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t e_ = (expr);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            cudaGetLastError();  /* a returned error also sits in the last-error slot */ \
            throw ::rcg::Error{-2, std::string(#expr) + ": " + cudaGetErrorString(e_) + RCG_WHERE}; \
        }                                                                           \
    } while (0)

#define RCG_CHECK_LAUNCH()                                                          \
    do {                                                                            \
        cudaError_t e_ = cudaGetLastError();                                        \
        if (e_ != cudaSuccess)                                                      \
            throw ::rcg::Error{-2, std::string("kernel launch: ") + cudaGetErrorString(e_) + RCG_WHERE}; \
    } while (0)

// Launch counter shared by all launchers of a context (set by the caller).
extern thread_local long long *g_launch_counter;
// Bound of the tensor-core kernels' main-loop waits for the calling context
// (rcg_options.spin_budget; 0 = the built-in bound), set around each call.
extern thread_local long long g_spin_budget;
inline void count_launch() { if (g_launch_counter) ++*g_launch_counter; }

// ------------------------------------------------------------ grid / operator
// Matrix-free description of A~_s (see include/rcg.h): x fastest, the z axis
// (last) carries the Robin faces, y is absent in 2D (Ny == 1).
struct Grid {
    int Nx, Ny, Nz;
    long long n;       // Nx*Ny*Nz
    long long ld;      // padded column stride of every n-vector (elements)
    // Diffusion tracking the absorption (rcg_options.d_model): the per-sample
    // D (float64 / float32) and face weights (3 columns) of sample slot s sit
    // at s ld (D) and 3 s ld (W) from these bases.  A kernel handed the
    // diagonal of slot s (dbase + s ld, the only diagonals the library passes)
    // finds that slot's coefficients at the same offset.  Null: fixed D.
    const double *dbase64 = nullptr, *Ds64 = nullptr, *Ws64 = nullptr;
    const float *dbase32 = nullptr, *Ds32 = nullptr;
    long long dspan = 0;                 // slots x ld: offsets past it are not a sample's
};

// The D of the sample whose diagonal is dg (tracking), else the shared D.
__host__ __device__ inline const double *sample_D(const Grid &g, const double *dg, const double *D) {
    if (!g.Ds64) return D;
    const long long o = dg - g.dbase64;
    return (o >= 0 && o < g.dspan) ? g.Ds64 + o : D;
}
__host__ __device__ inline const float *sample_D(const Grid &g, const float *dg, const float *D) {
    if (!g.Ds32) return D;
    const long long o = dg - g.dbase32;
    return (o >= 0 && o < g.dspan) ? g.Ds32 + o : D;
}
// The face weights (3 columns, stride ld) of the sample whose float64 diagonal is dg.
__host__ __device__ inline const double *sample_W(const Grid &g, const double *dg, const double *W) {
    if (!g.Ws64) return W;
    const long long o = dg - g.dbase64;
    return (o >= 0 && o < g.dspan) ? g.Ws64 + 3 * o : W;
}

// Columns addressed as base + j*ld.
template <typename T> struct Cols {
    T *p;
    long long ld;
    __host__ __device__ T *col(int j) const { return p + (long long)j * ld; }
};

constexpr int KMAX = 48;        // stride of the per-lane deflation arrays
constexpr int KU_MAX = 16;      // shared (seed eigenvector) deflation columns
constexpr int KP_MAX = RCG_MAX_PRIVATE;   // private deflation columns per lane

// Per-lane CG state on the device (structure of arrays, m lanes).
struct LaneState {
    int m;                  // lane capacity (stride of the ring buffers)
    int nl;                 // lanes 0 .. nl-1 of the current wave (<= m): launch extent
    double *rr;             // [3][m]  r^T r ring (slot = iteration mod 3)
    double *pq;             // [2][m]  p^T A p ring
    double *wv;             // [2][m][KMAX] (A W)^T r ring
    double *gw;             // [m][KMAX][KMAX] Cholesky factor of W^T A W (lower)
    int *kdef;              // [m] deflation columns of the lane
    int *active;            // [m] 1 while the lane iterates
    int *flag;              // [m] set to 1 when the recursive residual met thresh
    int *iters;             // [m]
    double *thresh;         // [m] stop threshold on ||r|| of the current cycle
    unsigned long long *prof;  // optional work counters (see KTimer), or null
    float *xa;              // [m] alpha of the step x += alpha p still to apply (float32 iteration)
    int *xt;                // [m] iteration that set xa (-1: none); applied by that iteration's direction kernel
    int maxit;              // iteration budget of a lane (recycled MINRES lanes)
};

// Per-lane scalars of the recycled MINRES lanes (minres.cu), [m][MR_NSC].
enum {
    MR_XI2, MR_XI, MR_PHI, MR_BETA, MR_C1, MR_S1, MR_C2, MR_S2, MR_WN2, MR_TAU, MR_GAMMA, MR_DELTA, MR_EPS,
    MR_IBETA, MR_THRESH, MR_NSC = 16
};

// Slots of a lane's private deflation columns in LaneGeom::wpp (the private
// columns plus one for the learned column).
constexpr int KPT = KP_MAX + 1;

// Addressing of the lanes of a wave (all columns ld apart):
//   x, r, p, q : lane l at base + l*ld (engine precision T)
//   deflation columns of lane l: c < k_u shared: W = wu + c*ld (the first
//   k_u basis columns), A W = awu + (si[l]*k_u + c)*ld (per sample slot);
//   c >= k_u private: W = wpp[l*KPT + c - k_u] (a pointer table: the columns
//   live in V, X_0 or the learned-column buffer, not copied per lane),
//   A W = awp + (l*kp_max + c - k_u)*ld.
struct LaneGeom {
    long long ld;
    int k_u, kp_max;
    int kp_sel;             // bound on every lane's current private count (<= kp_max): picks the kernels' templates
    void *x, *r, *p, *q;
    const void *wu, *awu, *awp;
    const void *const *wpp;
    const int *si, *kp;
};

// Optional per-launch device timing of the kernels of a CG iteration, with
// CUDA events on the launching stream.  Slots: 0 stencil, 1 update, 2 shared
// deflation dots, 3 per-lane scalars, 4 direction.  Work counters on the
// device (LaneState::prof): [0] stencil column applications, [1] update
// lanes, [2] update deflation columns, [3] direction lanes, [4] direction
// deflation columns.
struct KTimer {
    static constexpr int NK = 5;
    struct Rec { int slot; cudaEvent_t a, b; };
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> pending;
    double ms[NK] = {0, 0, 0, 0, 0};
    long long launches[NK] = {0, 0, 0, 0, 0};
    cudaEvent_t get() {
        if (pool.empty()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) throw Error{-2, "cudaEventCreate"};
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    // bracket a launch: e = start(st) before it, stop(slot, e, st) after it
    cudaEvent_t start(cudaStream_t st) {
        cudaEvent_t e = get();
        if (cudaEventRecord(e, st) != cudaSuccess) throw Error{-2, "cudaEventRecord"};
        return e;
    }
    void stop(int slot, cudaEvent_t a, cudaStream_t st) {
        cudaEvent_t b = get();
        if (cudaEventRecord(b, st) != cudaSuccess) throw Error{-2, "cudaEventRecord"};
        pending.push_back(Rec{slot, a, b});
    }
    // call after the stream is synchronised
    void harvest() {
        for (auto &r : pending) {
            float t = 0;
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) { ms[r.slot] += t; ++launches[r.slot]; }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
    }
    void reset() { harvest(); for (int k = 0; k < NK; ++k) { ms[k] = 0; launches[k] = 0; } }
    ~KTimer() {
        for (auto &r : pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Active lanes of a wave: `alist` (na lane indices, ascending) and tiles of
// at most 32 of them sharing a sample slot (tile_lane [ntiles][32]).
struct LaneList {
    const int *alist;
    int na;
    const int *tile_lane, *tile_si, *tile_cnt;
    int ntiles;
    // the lanes' p columns as one array (lane l at pbase + l pld, pcols
    // columns) and the sample diagonals (slot s at gbase + s Grid::ld,
    // gslots slots): the TMA stencil's tensor maps; null: not known
    const float *pbase = nullptr;
    long long pld = 0;
    int pcols = 0;
    const float *gbase = nullptr;
    int gslots = 0;
};

// ------------------------------------------------------------ learned augmentation (cnn.cu)
struct CnnGeom {
    int Nx, Ny, Nz;      // fine grid
    int f;               // pooling factor (4, 2 or 1; y is not pooled in 2D)
    int Gx, Gy, Gz;      // coarse grid
    long long V;         // coarse nodes
};
CnnGeom cnn_geom(const Grid &g);
int cnn_nparams();

// The network itself: a 3-level U-Net (16-32-64 channels, ten 3x3x3
// convolutions) on the coarse grid, bfloat16 activations on the tensor
// cores (unet.cu).  Layer l reads UNET_CIN[l] channels (stacked
// [up(deeper), skip] for layers 5 and 7) and writes UNET_COUT[l].
constexpr int UNET_LAYERS = 10;
extern const int UNET_CIN[UNET_LAYERS];
extern const int UNET_COUT[UNET_LAYERS];

class UNet {
  public:
    UNet(int Gx, int Gy, int Gz);
    ~UNet();
    UNet(const UNet &) = delete;
    UNet &operator=(const UNet &) = delete;
    // bfloat16 copies of the weights in the kernels' layouts (forward, and the
    // transposed layout of the backward pass when `backward`)
    void pack(cudaStream_t st, const float *theta, bool backward);
    // in[B][2][V0] -> out[B][V0] (float32); biases read from theta
    void forward(cudaStream_t st, const float *theta, const float *in, int B, float *out);
    // grad[P] (zeroed here) from d loss / d out [B][V0], after forward() on the same batch
    void backward(cudaStream_t st, const float *dout, int B, float *grad);
    // RCG_ERR_TIMEOUT if a tensor-core wait ran out since the last call (synchronises)
    int error(cudaStream_t st);
    // device bytes of the activations of one item
    long long bytes_per_item() const { return 2LL * (80 * V[0] + 144 * V[1] + 96 * V[2]) + 12 * 128; }

    int P = 0;
    int woff[UNET_LAYERS], boff[UNET_LAYERS];

  private:
    enum { A_IN, A_A0, A_S0, A_P0, A_A1, A_S1, A_P1, A_A2, A_A3, A_A4, A_A5, A_A6, A_N };
    struct Layer {
        int lvl, Cin, Cout, NP, NPb, Cg, nsrc;
        int sC[2] = {0, 0}, sreal[2] = {0, 0}, sup[2] = {0, 0}, sk0[2] = {0, 0}, sci0[2] = {0, 0};
        int nchunk, nchunk_b;
        long long pack_f, pack_b;
    };
    void layout(int B);
    void grow(void *&p, long long &cap, long long bytes);
    void conv(cudaStream_t st, int l, const __nv_bfloat16 *s0, const __nv_bfloat16 *s1, const float *bias, bool relu,
              __nv_bfloat16 *y, float *yf, const __nv_bfloat16 *mask, int B, bool backward = false,
              const __nv_bfloat16 *wp_override = nullptr);
    void down(cudaStream_t st, const __nv_bfloat16 *x, int C, int lvl, int B, __nv_bfloat16 *y);
    const __nv_bfloat16 *act(int id) const;
    __nv_bfloat16 *actw(int id);

    int G[3][3];
    long long V[3];
    Layer lay[UNET_LAYERS];
    long long aoff[A_N];
    void *wpf = nullptr, *wpb = nullptr, *abuf = nullptr, *gbuf = nullptr, *fbuf = nullptr;
    long long abuf_cap = 0, gbuf_cap = 0, fbuf_cap = 0;
    int *d_err = nullptr;
};

// The network, its Adam state, the recorded training pairs and work buffers
// (device memory owned here).
class Cnn {
  public:
    explicit Cnn(const Grid &g);
    ~Cnn();
    Cnn(const Cnn &) = delete;
    Cnn &operator=(const Cnn &) = delete;

    void set_weights(cudaStream_t st, const float *host);
    void refresh_bf16(cudaStream_t st);
    void features(cudaStream_t st, const float *const *r0, const double *const *mu, int nl, float *out);
    void forward(cudaStream_t st, const float *in, int B, float *out);
    double gradient(cudaStream_t st, const float *in, const float *tg, int B);
    void add_pairs(cudaStream_t st, const float *feat, const float *tgt, int cnt);
    double train(cudaStream_t st, int epochs, int B, double lr, unsigned long long seed);
    void upsample(cudaStream_t st, const float *out, float *const *dst, const int *rows, int B);
    void pool64(cudaStream_t st, const double *const *src, float *out, int B, float sign, bool accumulate);
    void normalise(cudaStream_t st, float *a, int B);
    void ensure(float *&p, long long &cap, long long need);

    CnnGeom geom;
    int P;
    bool have = false;       // weights set or trained
    bool record = false;     // record (features, target) pairs from solves
    int npairs = 0;
    float *theta = nullptr, *theta16 = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    double *d_loss = nullptr;
    long long t_adam = 0;
    UNet net;
    // work buffers of the solver integration (grown on demand)
    float *feat = nullptr, *outc = nullptr, *x0c = nullptr;
    long long feat_cap = 0, outc_cap = 0, x0c_cap = 0;

  private:
    void forward_backward(cudaStream_t st, const float *in, const float *tg, int B);
    float *act = nullptr;
    long long act_cap = 0;
    float *pin = nullptr, *ptg = nullptr;
    long long pair_cap = 0;
    float *bin = nullptr, *btg = nullptr;
    long long bin_cap = 0, btg_cap = 0;
    int *d_idx = nullptr;
    long long idx_cap = 0;
};

// Augmentation of the private deflation spaces by the network's columns:
// dots of A~ x_hat with every deflation column and x_hat, then the Galerkin
// pivot test and the bordered inverse (see cnn.cu).
void aug_dots(cudaStream_t st, long long n, long long ld, const float *V, int ku, const float *const *wpp,
              const float *awp, int kps, const int *kp, const int *alist, int na, double *cd);
void aug_border(cudaStream_t st, double *gw, int *kdef, int *kp, const int *alist, int na, const double *cd,
                double tau, int *kept);

// ------------------------------------------------------------ launchers
// stencil.cu
template <typename T>
void apply_op(cudaStream_t st, const Grid &g, const T *D, const T *const *diag_of_col,
              const T *const *src, T *const *dst, int ncols, const int *active,
              double *dots, unsigned long long *act_count = nullptr);
void face_weights(cudaStream_t st, const Grid &g, const double *D, double *W);
void residual64(cudaStream_t st, const Grid &g, const double *W, const double *const *diag_of_col,
                const double *const *x, double *const *r, float *const *r32, int ncols,
                const int *node, const double *bw, double *rr, const int *active, int nact = -1);

// track.cu (diffusion tracking the absorption)
void track_coefficients(cudaStream_t st, const Grid &g, const double *mu, double mus, double h, double robin_A,
                        double *D64, float *D32, double *W64, double *diag64, float *diag32);
void track_deriv(cudaStream_t st, const Grid &g, const double *D, const double *dmu, double h, double robin_A,
                 double scale, double *dg, double *dw);
void track_touch(cudaStream_t st, const Grid &g, const double *dg, const double *dw, double *touch);
template <typename T>
void delta_rows(cudaStream_t st, const Grid &g, const int *blist, int b0, int nb, const double *dg, const double *dw,
                const T *X, long long ldx, int ncols, T *Xc, double *Yc, long long ldc);
void rhs_weights(cudaStream_t st, const double *D, const int *node, const double *wt, int nsrc, int nrhs,
                 double robin_A, double h, double *w, const double *dmu = nullptr, long long lddmu = 0,
                 int nparam = 0, double *dwt = nullptr);
void jac_rhs_terms(cudaStream_t st, int nparam, int nd, int ns, const double *dwt, const double *Pd, const double *Ps,
                   double *J);
void ratio_scale(cudaStream_t st, long long n, const double *x, long long ldx, const double *w1, const double *w0,
                 double *dst, long long ldd, int ncols);

// dense.cu
template <typename TA, typename TB>
void gemm_tn(cudaStream_t st, long long n, const TA *A, long long lda, int ka,
             const TB *B, long long ldb, int kb, double *C, int ldc, bool accumulate,
             const double *wt = nullptr, const int *rows = nullptr, long long nrows = 0);
void gemm_tn_df(cudaStream_t st, long long n, const float *A, long long lda, int ka, const double *B, long long ldb,
                int kb, double *C, int ldc, bool accumulate);
// J_qk = Z_q^T G_qk X_q for k < nparam, q < nq (G: [q][k] r x r symmetric,
// X_q = X + q r ns, Z_q = Z + q r nd, ld r; J_qk = J + (q nparam + k) nd ns)
void rom_jac(cudaStream_t st, int r, int nparam, const double *G, const double *X, int ns, const double *Z, int nd,
             double *J, int nq = 1);
// dst[c] <- src[c] (n elements) for c < cnt, one launch (device pointer lists;
// 16-byte aligned columns)
template <typename T>
void copy_cols(cudaStream_t st, long long n, const T *const *src, T *const *dst, int cnt);
// Psi_q = Crm^T X_q (nd x ns) for q < nq (Crm r x nd, X_q = X + q r ns, ld r)
void rom_psi(cudaStream_t st, int r, int nq, const double *Crm, const double *X, int ns, int nd, double *Psi);
template <typename TA, typename TB, typename AT>
void gemm_tn_acc(cudaStream_t st, long long n, const TA *A, long long lda, int ka,
                 const TB *B, long long ldb, int kb, double *C, int ldc, bool accumulate,
                 const double *wt = nullptr, const int *rows = nullptr, long long nrows = 0);
// tc.cu: C (+)= A^T B for float32 A, B on the tensor cores (3xTF32)
long long tc_gemm_tn_scratch(long long n, int ka, int kb, bool symmetric, int *z_out, long long *chunk_out);
bool tc_gemm_tn_ok(long long lda, long long ldb, const void *A, const void *B);
void tc_gemm_tn(cudaStream_t st, long long n, const float *A, long long lda, int ka, const float *B, long long ldb,
                int kb, double *C, int ldc, bool accumulate, bool symmetric, float *scratch, int *err,
                const double *wt = nullptr, const int *blist = nullptr, const int *bcount = nullptr);
// C_b = A^T diag(w_b) A for nbatch weight vectors in one launch (see tc.cu).
long long tc_gram_w_batched_scratch(int ka, int nbatch, int *zper_out);
void tc_gram_w_batched(cudaStream_t st, long long n, const float *A, long long lda, int ka, double *C, int ldc,
                       long long ldcb, int nbatch, const double *wt, long long ldw, const int *blist, long long ldl,
                       const int *bcount, float *scratch, int *err, bool accumulate = false, double wscale = 1.0);
long long tc_gemm_nn_scratch(int k, int m);
void tc_gemm_nn(cudaStream_t st, long long n, const float *V, long long ldv, int k, const double *C, int ldc, int m,
                float *Out, long long ldo, double alpha, double beta, float *scratch, int *err);
// Blocks of 32 rows where w does not vanish, for nvec weight vectors (w + v ldw
// -> list + v ldl, count[v]).
void tc_block_list(cudaStream_t st, long long n, const double *w, int *list, int *count, int nvec = 1,
                   long long ldw = 0, long long ldl = 0);
template <typename TA, typename TO>
void gemm_nn(cudaStream_t st, long long n, const TA *A, long long lda, int k,
             const double *Y, int ldy, int m, TO *Out, long long ldo, double alpha, double beta);
void gemm_nn_df(cudaStream_t st, long long n, const float *V, long long ldv, int k, const double *Y, int ldy,
                int m, double *Out, long long ldo, double beta);
template <typename TV>
void gather_rows(cudaStream_t st, const TV *V, long long ldv, int r, const int *node,
                 const double *w, int m, double *out, int ldo);
template <typename TS, typename TD>
void convert_cols(cudaStream_t st, long long n, const TS *src, long long lds, TD *dst,
                  long long ldd, int ncols);
template <typename T>
void col_dots(cudaStream_t st, long long n, const T *A, long long lda, const T *B,
              long long ldb, int ncols, double *out);
void add_cols_f32_to_f64(cudaStream_t st, long long n, double *x, long long ldx, const float *d,
                         long long ldd, const int *lanes, int nl);

// small.cu (float64, small dense matrices)
void chol_inplace(cudaStream_t st, double *A, int lda, int r, int *info);
void chol_border(cudaStream_t st, double *L, int ldl, int r_old, int a, int *info);
void trsv_lower_batched(cudaStream_t st, const double *L, int ldl, int r, double *B, int ldb,
                        int m, bool transpose);
// nbatch independent systems: factor b at A + b strideA (failure: *info = max first bad pivot + 1)
void chol_batched(cudaStream_t st, double *A, int lda, long long strideA, int r, int nbatch, int *info);
// nbatch factors L + b strideL, each with m right-hand sides B + b strideB
void trsv_multi(cudaStream_t st, const double *L, int ldl, long long strideL, int r, double *B, int ldb,
                long long strideB, int m, int nbatch, bool transpose);
void ordered_drop_chol(cudaStream_t st, const double *M, int a, const double *xnorm2, double *S,
                       double tau, double *R, int *kept, double *ratio);
void tri_upper_inverse(cudaStream_t st, const double *R, int ldr, int a, double *Ri);
void lane_inverse(cudaStream_t st, double *gw, const int *kdef, int m, int *info);
void jacobi_eig(cudaStream_t st, double *A, int lda, int k, double *Q, double *w);
// parallel cyclic Jacobi (m2 even): eigenvalues on diag(A), eigenvectors in Q; returns sweeps
int jacobi_parallel(cudaStream_t st, double *A, int lda, int m2, double *Q, int ldq, double *cs, double *red,
                    double tol, int max_sweeps);

// misc.cu
void diag_star(cudaStream_t st, const Grid &g, const double *D, double h, double A, double *out);
void diag_sample(cudaStream_t st, long long n, const double *dstar, const double *mu, double h2,
                 double *d64, float *d32);
void scaled_diff(cudaStream_t st, long long n, const double *a, const double *b, double scale, double *w);
template <typename TS, typename TD>
void convert_lanes(cudaStream_t st, long long n, const TS *const *src, const int *lanes, int nl,
                   TD *dst, long long ldd);
void norm2_lanes(cudaStream_t st, long long n, const double *const *src, const int *lanes, int nl,
                 double *out);
void border_write(cudaStream_t st, double *C, int ldc, int r0, int a, const double *B, int ldb);
void copy_new_rows(cudaStream_t st, const double *G, double *L, int ld, int r0, int a);
void gather_sub(cudaStream_t st, const double *R, int a, const int *K, int ak, double *RK);
void scatter_rows(cudaStream_t st, const double *Rinv, int ak, const int *K, int a, double *Rhat);
void lower_to_upper(cudaStream_t st, const double *L, int lda, int a, double *R);
void lane_gw(cudaStream_t st, const double *const *Gs, int ldg, int r, const int *spec,
             const double *const *sx, const int *kdef, double *gw, int m);

template <typename T>
void rand_fill(cudaStream_t st, T *X, long long n, long long ld, int b, unsigned long long seed);
template <typename T>
void cheb_step(cudaStream_t st, T *out, const T *AY, const T *Y, const T *Yp, long long n, long long ld,
               int b, double alpha, double beta, double gamma);
void gershgorin(cudaStream_t st, const Grid &g, const double *D, const double *diag, unsigned long long *out);
template <typename T>
void ritz_res(cudaStream_t st, const T *AX, const T *X, const double *theta, long long n, long long ld,
              int b, double *res2);

// cg4.cu (float32, Nx % 4 == 0)
bool cg4_supported(const Grid &g);
bool stencil4z_supported(const Grid &g);
void cg_iteration4(cudaStream_t st, const Grid &g, const float *D, const float *const *diag_of_col,
                   const float *const *p_ptr, float *const *q_ptr, LaneGeom gm, LaneState ls, LaneList ll, int t,
                   float *mu, float *beta, KTimer *kt);
void cg_restart4(cudaStream_t st, const Grid &g, LaneGeom gm, LaneState ls, LaneList ll, int t, float *mu,
                 float *beta, int *drop = nullptr);
void lane_zero(cudaStream_t st, LaneState ls, const int *mask);
// q = A~_s p on ncols float32 columns with the inner iteration's stencil
// variant v (-1: the autotuned choice; see cg4.cu), p^T q added into
// dots[lanes[c]]; `active[lanes[c]]` != 0 for the columns to apply.
void stencil4_apply(cudaStream_t st, const Grid &g, const float *D, const float *const *diag, const float *const *p,
                    float *const *q, int ncols, const int *lanes, const int *active, double *dots, int v,
                    const float *pbase = nullptr, long long pld = 0, const float *gbase = nullptr, int gslots = 0);
// RCG_ERR_TIMEOUT if a TMA stencil's wait ran out since the last call (synchronises the stream), else 0
int stencil_take_error(cudaStream_t st);
std::string stencil_tuning_report();
const char *stencil_variant_name(int v);
int stencil_variant_ok(const Grid &g, int v);

// minres.cu (float64 lanes; LaneGeom as for CG with x = the MINRES iterate
// y, p = v_k, q = A~ v_k / w; ext = [m][3] extra columns v_{k-1}, d_{k-1}, d_{k-2})
// Gram / dots of the lane's recycle columns: A~W (use_w false) or W itself
void mres_gram(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const int *mask, double *H,
               bool use_w = false);
void mres_dots(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const int *mask,
               const double *src, double *hd, bool use_w = false);
// dst = src - W mu (lane blocks), ||dst||^2 added into sc[MR_XI2]
void mres_sub(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const int *mask,
              const double *src, const double *mu, double *dst, double *sc);
void mres_mu(cudaStream_t st, const LaneState &ls, const int *mask, const double *hd, double *mu, double *sc);
void mres_cycle(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const int *mask,
                const double *mu, double *const *x64, double *sc, bool finish);
void mres_init(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const int *mask, double *ext,
               double *sc, int *act);
void mres_iteration(cudaStream_t st, const Grid &g, const double *D, const double *const *diag_of_col,
                    const double *const *v_ptr, double *const *q_ptr, const LaneGeom &gm, const LaneState &ls,
                    int *act, int *step, double *alpha, double *hd, double *mu, double *ext, double *sc);

// cg.cu
template <typename T>
void cg_iteration(cudaStream_t st, const Grid &g, const T *D, const T *const *diag_of_col,
                  const T *const *p_ptr, T *const *q_ptr, LaneGeom gm, LaneState ls, int t,
                  KTimer *kt = nullptr);
template <typename T>
void cg_restart(cudaStream_t st, const Grid &g, LaneGeom gm, LaneState ls, int t, const int *mask,
                int *drop = nullptr);
// Lanes with drop[l] != 0 lose their last private deflation column (kdef, kp - 1); drop is cleared.
void drop_last_private(cudaStream_t st, LaneState ls, int *kp, int *drop, int m);
template <typename T>
void gather_cols(cudaStream_t st, long long n, const T *const *src, T *dst, long long ld, int count);

}  // namespace rcg
