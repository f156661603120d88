// librcg host runtime: the C ABI of include/rcg.h, device memory of a
// context, and the driver of Algorithm 2 (Sec. 4.3) over the kernels.
//
// A "wave" is a set of (sample, RHS) lanes handled together with the basis V
// frozen: the Galerkin check from range(V), batched deflated CG on the lanes
// whose check failed (with FP64 refinement restarts), and one ordered
// rank-revealing append of their solutions.  RCG_SEQUENTIAL runs one lane
// per wave in the paper's order (V grows between right-hand sides);
// RCG_WAVE puts all RHS of `wave_samples` samples into one wave.
#include "common.cuh"
#include "../../include/rcg.h"

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

using namespace rcg;

namespace {

template <typename TS>
__global__ void k_add_lanes(long long n, double *__restrict__ x, long long ldx, const TS *__restrict__ d,
                            long long ldd, const int *__restrict__ lanes) {
    const int l = lanes[blockIdx.y];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        x[(long long)l * ldx + p] += (double)d[(long long)l * ldd + p];
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
};

// A chunk of CG iterations captured once as a CUDA graph and replayed on the
// context's stream.  Capture needs a stream other than the legacy default
// one, so the graph runs on a private stream ordered after / before the
// context's stream by events.  Launches issued during the capture are counted
// once per replay.
class CgGraph {
  public:
    explicit CgGraph(cudaStream_t st) : st_(st) {}
    CgGraph(const CgGraph &) = delete;
    CgGraph &operator=(const CgGraph &) = delete;
    ~CgGraph() {
        if (exec_) cudaGraphExecDestroy(exec_);
        if (graph_) cudaGraphDestroy(graph_);
        if (ev0_) cudaEventDestroy(ev0_);
        if (ev1_) cudaEventDestroy(ev1_);
        if (gs_) cudaStreamDestroy(gs_);
    }
    bool ready() const { return exec_ != nullptr; }
    template <typename F> void capture(F issue) {
        RCG_CUDA_TRY(cudaStreamCreateWithFlags(&gs_, cudaStreamNonBlocking));
        RCG_CUDA_TRY(cudaEventCreateWithFlags(&ev0_, cudaEventDisableTiming));
        RCG_CUDA_TRY(cudaEventCreateWithFlags(&ev1_, cudaEventDisableTiming));
        long long *ctr = g_launch_counter;
        long long counted = 0;
        g_launch_counter = &counted;
        RCG_CUDA_TRY(cudaStreamBeginCapture(gs_, cudaStreamCaptureModeThreadLocal));
        try {
            issue(gs_);
        } catch (...) {
            cudaGraph_t dummy = nullptr;
            cudaStreamEndCapture(gs_, &dummy);
            if (dummy) cudaGraphDestroy(dummy);
            g_launch_counter = ctr;
            throw;
        }
        g_launch_counter = ctr;
        RCG_CUDA_TRY(cudaStreamEndCapture(gs_, &graph_));
        RCG_CUDA_TRY(cudaGraphInstantiate(&exec_, graph_, 0));
        per_launch_ = counted;
    }
    void launch() {
        RCG_CUDA_TRY(cudaEventRecord(ev0_, st_));
        RCG_CUDA_TRY(cudaStreamWaitEvent(gs_, ev0_, 0));
        RCG_CUDA_TRY(cudaGraphLaunch(exec_, gs_));
        RCG_CUDA_TRY(cudaEventRecord(ev1_, gs_));
        RCG_CUDA_TRY(cudaStreamWaitEvent(st_, ev1_, 0));
        if (g_launch_counter) *g_launch_counter += per_launch_;
    }

  private:
    cudaStream_t st_, gs_ = nullptr;
    cudaEvent_t ev0_ = nullptr, ev1_ = nullptr;
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    long long per_launch_ = 0;
};

// dst = x / sqrt(nrm2[0]) (a recycle column of unit length)
template <typename TD>
__global__ void k_scaled_copy(long long n, const double *__restrict__ x, const double *__restrict__ nrm2,
                              TD *__restrict__ dst) {
    const double s = nrm2[0] > 0.0 ? 1.0 / sqrt(nrm2[0]) : 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        dst[p] = (TD)(x[p] * s);
}

}  // namespace

// The state right after rcg_seed of an engine, for copying it into another
// context (device pointers owned by the source).
struct SeedView {
    bool seeded = false;
    int esize = 0;                     // bytes per element of V and X_0
    int r_seed = 0, k_u = 0, s_star = -1, rmax = 0;
    const void *V = nullptr, *X0 = nullptr;
    const double *Cstar = nullptr;
    std::vector<std::vector<int>> priv_seed;
};

struct EngineBase {
    virtual ~EngineBase() {}
    virtual SeedView seed_view() const = 0;
    virtual void seed_import(const SeedView &sv) = 0;
    virtual void seed(int s0, const double *U0, rcg_stat *stats) = 0;
    virtual void reset() = 0;
    virtual int compress(int r_cap, double tau, std::vector<double> &sigma) = 0;
    virtual int solve_all(int s_first, int s_count, rcg_stat *stats) = 0;
    virtual int rank() const = 0;
    virtual void basis_get(double *V) = 0;
    virtual void rom_eval(const double *mu, int nparam, const double *dmu, double *Psi, double *J) = 0;
    virtual void rom_eval_batch(int nq, const double *mu, int nparam, const double *dmu, double *Psi, double *J) = 0;
    virtual void sample_changed(int s) = 0;
    virtual void save(std::FILE *f) = 0;
    virtual void load(std::FILE *f) = 0;
};

// ---------------------------------------------------------- state file I/O
// Binary layout of rcg_save: magic, a header of int64 fields, then arrays
// (each: int64 count, raw elements).  Little-endian host order.
constexpr char kMagic[8] = {'R', 'C', 'G', 'S', 'T', 'A', 'T', '2'};
inline void wr(std::FILE *f, const void *p, size_t bytes) {
    if (bytes && std::fwrite(p, 1, bytes, f) != bytes) throw Error{RCG_ERR_INVALID, "rcg_save: write failed"};
}
inline void rd(std::FILE *f, void *p, size_t bytes) {
    if (bytes && std::fread(p, 1, bytes, f) != bytes) throw Error{RCG_ERR_INVALID, "rcg_load: truncated file"};
}
template <typename V> void wr_vec(std::FILE *f, const std::vector<V> &v) {
    const long long c = (long long)v.size();
    wr(f, &c, sizeof(c));
    wr(f, v.data(), sizeof(V) * v.size());
}
template <typename V> std::vector<V> rd_vec(std::FILE *f, long long max_count) {
    long long c = 0;
    rd(f, &c, sizeof(c));
    if (c < 0 || c > max_count) throw Error{RCG_ERR_INVALID, "rcg_load: bad array length"};
    std::vector<V> v((size_t)c);
    rd(f, v.data(), sizeof(V) * v.size());
    return v;
}

struct rcg_ctx {
    rcg_grid grid{};
    rcg_options opt{};
    cudaStream_t st = nullptr;
    Grid g{};
    long long n = 0, ld = 0;
    double h = 0;
    std::string err;
    long long launches = 0;
    std::vector<void *> allocs;
    size_t bytes = 0;
    // host mirrors
    bool have_D = false, have_rhs = false;
    int nsrc = 0, ndet = 0, nrhs = 0;
    std::vector<int> rhs_node;
    std::vector<double> rhs_w, rhs_wt, tol;   // effective weights at the reference D; source / detector strengths
    std::vector<char> sample_set;
    // device coefficient fields
    double *D64 = nullptr, *dstar = nullptr, *mu64 = nullptr, *diag64 = nullptr;
    // diffusion tracking the absorption: per-sample D, face weights (3 columns)
    double *Ds64 = nullptr, *Ws64 = nullptr;
    float *Ds32 = nullptr;
    bool track() const { return opt.d_model == RCG_D_TRACKS_MU; }
    double *Ds64_of(int s) { return Ds64 + (long long)s * ld; }
    double *Ws64_of(int s) { return Ws64 + 3LL * s * ld; }
    double *W64 = nullptr;             // face weights (D_p + D_q)/2 towards +x, +y, +z (3 columns)
    float *D32 = nullptr, *diag32 = nullptr;
    int *d_rhs_node = nullptr;
    double *d_rhs_w = nullptr, *d_rhs_wt = nullptr, *d_ones = nullptr;
    std::unique_ptr<EngineBase> eng;
    std::map<std::string, double> phase;
    std::vector<std::vector<double>> solutions;   // per sample, host copies (keep_solutions)
    KTimer ktimer;                                 // optional device timing of the CG kernels
    std::unique_ptr<Cnn> cnn;                      // learned augmentation (created on first use)
    Cnn &net() {
        if (!cnn) cnn.reset(new Cnn(g));
        return *cnn;
    }
    unsigned long long *d_prof = nullptr;          // work counters of the CG kernels

    template <typename T> T *alloc(size_t count) {
        void *p = nullptr;
        const size_t b = std::max<size_t>(count, 1) * sizeof(T);
        if (cudaMalloc(&p, b) != cudaSuccess) {
            cudaGetLastError();
            throw Error{RCG_ERR_OOM, "cudaMalloc of " + std::to_string(b) + " bytes failed"};
        }
        allocs.push_back(p);
        bytes += b;
        return (T *)p;
    }
    void release(void *p) {
        if (!p) return;
        auto it = std::find(allocs.begin(), allocs.end(), p);
        if (it != allocs.end()) { allocs.erase(it); cudaFree(p); }
    }
    void sync() { RCG_CUDA_TRY(cudaStreamSynchronize(st)); }
    template <typename T> void h2d(T *d, const T *h, size_t count) {
        RCG_CUDA_TRY(cudaMemcpyAsync(d, h, count * sizeof(T), cudaMemcpyHostToDevice, st));
    }
    template <typename T> void d2h(T *h, const T *d, size_t count) {
        RCG_CUDA_TRY(cudaMemcpyAsync(h, d, count * sizeof(T), cudaMemcpyDeviceToHost, st));
    }
    double *diag64_of(int s) { return diag64 + (long long)s * ld; }
    float *diag32_of(int s) { return diag32 + (long long)s * ld; }
};

namespace {

// ------------------------------------------------------------------ engine
template <typename T>
struct Engine : EngineBase {
    rcg_ctx *c;
    cudaStream_t st;
    Grid g;
    long long n, ld;
    int rmax;
    const T *D;
    bool mixed;

    // basis and caches
    T *V = nullptr;
    int vcap = 0;                      // columns allocated for V (grows to rmax)
    int r = 0, r_seed = 0, s_star = -1, k_u = 0;
    double *Cstar = nullptr;           // V^T A~_* V, ld rmax
    T *X0 = nullptr;                   // seed solutions (nrhs columns)
    double *sX0 = nullptr;             // V^T X0, ld rmax
    bool seeded = false;
    std::vector<std::vector<int>> priv, priv_seed;   // per RHS: V indices, -1 = X0 column
    // sequential Galerkin state (current sample)
    int gs_sample = -1, gs_r = 0;
    double *Gs = nullptr, *Ls = nullptr;
    // per-sample wave Galerkin matrices and Delta weights
    std::vector<double *> Gw, Lw, dw;
    std::vector<int> dw_star;
    std::vector<int *> dwl;            // per sample: 32-row blocks where Delta does not vanish
    int *dwc = nullptr;                // their counts (device, one per sample slot)
    int *rom_bl = nullptr, *rom_bc = nullptr;
    // reduced Jacobian: per-parameter weights, block lists, G_k and G_k X_r
    double *jk_w = nullptr, *jk_G = nullptr;
    long long jk_gcap = 0;
    int *jk_bl = nullptr, *jk_bc = nullptr;
    // rom_eval_batch: per-point reduced matrices, weights, block lists, solves, Jacobian Grams
    double *rb_A = nullptr, *rb_w = nullptr, *rb_X = nullptr, *rb_Z = nullptr, *rb_G = nullptr;
    int *rb_bl = nullptr, *rb_bc = nullptr, *rb_jbl = nullptr, *rb_jbc = nullptr;
    long long rb_cap[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int jk_cap = 0;
    // lanes workspace
    int mcap = 0;
    double *x64 = nullptr;
    T *xc = nullptr, *rv = nullptr, *pv = nullptr, *qv = nullptr;
    LaneState ls{};
    int *d_mask = nullptr, *d_lnode = nullptr, *d_list = nullptr;
    double *d_lw = nullptr, *d_rr = nullptr;
    double **p_x64 = nullptr, **p_diag64 = nullptr;
    T **p_xc = nullptr, **p_r = nullptr, **p_p = nullptr, **p_q = nullptr, **p_diag = nullptr;
    int *d_spec = nullptr, *d_si = nullptr, *d_kp = nullptr;
    double **d_sx = nullptr, **d_gsl = nullptr;
    const void **d_wpp = nullptr;      // private deflation columns of each lane, [m][KPT] addresses
    T *xhb = nullptr;                  // the network's columns of a wave
    int xhb_cap = 0;
    float *mu_f = nullptr, *beta_f = nullptr;      // per-lane mu, beta of the float32 iteration
    int *d_alist = nullptr, *d_tlane = nullptr, *d_tsi = nullptr, *d_tcnt = nullptr;
    double *Yb = nullptr;
    // deflation A W buffers
    T *au0 = nullptr;
    int au0_cap = 0, au0_ku = -1, au0_star = -1;
    bool au0_valid = false;
    std::vector<int> au0_samples;
    T *awp = nullptr;
    long long awp_cap = 0;
    // pointer scratch for generic applies
    const void **d_ptrA = nullptr, **d_ptrB = nullptr, **d_ptrC = nullptr;
    int ptr_cap = 0;
    // append workspace
    int acap = 0;
    T *Wb = nullptr, *Qb = nullptr;
    double *Cb = nullptr, *M = nullptr, *S = nullptr, *R = nullptr, *RK = nullptr, *Ri = nullptr, *Rhat = nullptr;
    double *xn2 = nullptr, *ratio_d = nullptr;
    int *kept_d = nullptr, *d_K = nullptr, *d_cand = nullptr;
    int *d_info = nullptr;          // [0] Cholesky info, [1] sticky tensor-core wait timeout
    float *tc_scr = nullptr;        // split-K slices of the tensor-core products
    long long tc_cap = 0;
    // learned augmentation: per-lane pointer lists, rows, pivot data
    const float **d_lr = nullptr;
    const double **d_lm = nullptr, **d_lx = nullptr;
    float **d_ldst = nullptr;
    int *d_arow = nullptr, *d_aug_l = nullptr, *d_kept = nullptr, *d_drop = nullptr;
    double *d_cd = nullptr;
    int lp_cap = 0;
    void ensure_learn(int m) {
        if (m <= lp_cap) return;
        for (void *p : std::vector<void *>{(void *)d_lr, (void *)d_lm, (void *)d_lx, (void *)d_ldst, (void *)d_arow,
                                           (void *)d_aug_l, (void *)d_kept, (void *)d_drop, (void *)d_cd})
            c->release(p);
        lp_cap = m;
        d_lr = c->alloc<const float *>(m);
        d_lm = c->alloc<const double *>(m);
        d_lx = c->alloc<const double *>(m);
        d_ldst = c->alloc<float *>(m);
        d_arow = c->alloc<int>(m);
        d_aug_l = c->alloc<int>(m);
        d_kept = c->alloc<int>(m);
        d_drop = c->alloc<int>(m);
        d_cd = c->alloc<double>((size_t)m * (KMAX + 1));
    }
    // rom workspace
    double *Ar = nullptr, *Br = nullptr, *Crm = nullptr, *Xr = nullptr, *Zr = nullptr, *wtmp = nullptr;
    double *VX = nullptr, *VZ = nullptr;

    explicit Engine(rcg_ctx *ctx) : c(ctx), st(ctx->st), g(ctx->g), n(ctx->n), ld(ctx->ld), rmax(ctx->opt.r_max) {
        mixed = sizeof(T) == 4;
        D = mixed ? (const T *)ctx->D32 : (const T *)ctx->D64;
        vcap = std::min(rmax, 512);
        V = c->alloc<T>((size_t)vcap * ld);
        Cstar = c->alloc<double>((size_t)rmax * rmax);
        Gs = c->alloc<double>((size_t)rmax * rmax);
        Ls = c->alloc<double>((size_t)rmax * rmax);
        d_info = c->alloc<int>(4);
        RCG_CUDA_TRY(cudaMemsetAsync(d_info, 0, 4 * sizeof(int), st));
        Gw.assign(c->opt.max_samples, nullptr);
        Lw.assign(c->opt.max_samples, nullptr);
        dw.assign(c->opt.max_samples, nullptr);
        dw_star.assign(c->opt.max_samples, -1);
        dwl.assign(c->opt.max_samples, nullptr);
        dwc = c->alloc<int>(c->opt.max_samples);
    }

    const T *diagT(int s) const { return mixed ? (const T *)c->diag32_of(s) : (const T *)c->diag64_of(s); }

    // --------------------------------------------------------- workspaces
    void ensure_lanes(int m) {
        if (m <= mcap) return;
        for (void *p : std::vector<void *>{x64, xc, rv, pv, qv, ls.rr, ls.pq, ls.wv, ls.gw, ls.kdef, ls.active, ls.flag,
                                           ls.iters, ls.thresh, ls.xa, ls.xt, d_mask, d_lnode, d_list, d_lw, d_rr,
                                           p_x64, p_diag64, p_xc, p_r, p_p, p_q, p_diag, d_spec, d_sx, d_gsl, Yb, d_si, d_kp,
                                           mu_f, beta_f, d_alist, d_tlane, d_tsi, d_tcnt, d_wpp})
            c->release(p);
        mcap = m;
        d_wpp = c->alloc<const void *>((size_t)m * KPT);
        x64 = c->alloc<double>((size_t)m * ld);
        xc = c->alloc<T>((size_t)m * ld);
        rv = c->alloc<T>((size_t)m * ld);
        pv = c->alloc<T>((size_t)m * ld);
        qv = c->alloc<T>((size_t)m * ld);
        ls.m = m;
        ls.nl = m;
        ls.rr = c->alloc<double>(3 * (size_t)m);
        ls.pq = c->alloc<double>(2 * (size_t)m);
        ls.wv = c->alloc<double>(2 * (size_t)m * KMAX);
        ls.gw = c->alloc<double>((size_t)m * KMAX * KMAX);
        ls.kdef = c->alloc<int>(m);
        ls.active = c->alloc<int>(m);
        ls.flag = c->alloc<int>(m);
        ls.iters = c->alloc<int>(m);
        ls.thresh = c->alloc<double>(m);
        ls.xa = c->alloc<float>(m);
        ls.xt = c->alloc<int>(m);
        d_si = c->alloc<int>(m);
        d_kp = c->alloc<int>(m);
        mu_f = c->alloc<float>((size_t)m * KMAX);
        beta_f = c->alloc<float>(m);
        d_alist = c->alloc<int>(m);
        d_tlane = c->alloc<int>((size_t)m * 32);
        d_tsi = c->alloc<int>(m);
        d_tcnt = c->alloc<int>(m);
        d_mask = c->alloc<int>(m);
        d_lnode = c->alloc<int>(m);
        d_list = c->alloc<int>(m);
        d_lw = c->alloc<double>(m);
        d_rr = c->alloc<double>(m);
        p_x64 = c->alloc<double *>(m);
        p_diag64 = c->alloc<double *>(m);
        p_xc = c->alloc<T *>(m);
        p_r = c->alloc<T *>(m);
        p_p = c->alloc<T *>(m);
        p_q = c->alloc<T *>(m);
        p_diag = c->alloc<T *>(m);
        d_spec = c->alloc<int>((size_t)m * KMAX);
        d_sx = c->alloc<double *>(m);
        d_gsl = c->alloc<double *>(m);
        Yb = c->alloc<double>((size_t)rmax * m);
        std::vector<double *> hx(m);
        std::vector<T *> hc(m), hr(m), hp(m), hq(m);
        for (int l = 0; l < m; ++l) {
            hx[l] = x64 + (long long)l * ld;
            hc[l] = xc + (long long)l * ld;
            hr[l] = rv + (long long)l * ld;
            hp[l] = pv + (long long)l * ld;
            hq[l] = qv + (long long)l * ld;
        }
        c->h2d(p_x64, hx.data(), m);
        c->h2d(p_xc, hc.data(), m);
        c->h2d(p_r, hr.data(), m);
        c->h2d(p_p, hp.data(), m);
        c->h2d(p_q, hq.data(), m);
        // lane state starts inactive over the whole capacity (fresh device memory
        // holds whatever an earlier allocation left there)
        RCG_CUDA_TRY(cudaMemsetAsync(ls.active, 0, sizeof(int) * m, st));
        RCG_CUDA_TRY(cudaMemsetAsync(ls.flag, 0, sizeof(int) * m, st));
        RCG_CUDA_TRY(cudaMemsetAsync(ls.kdef, 0, sizeof(int) * m, st));
        RCG_CUDA_TRY(cudaMemsetAsync(ls.iters, 0, sizeof(int) * m, st));
        RCG_CUDA_TRY(cudaMemsetAsync(ls.xt, 0xFF, sizeof(int) * m, st));
        RCG_CUDA_TRY(cudaMemsetAsync(d_mask, 0, sizeof(int) * m, st));
        // diagonal pointers of unused lanes point at a valid column (sample slot 0)
        {
            std::vector<double *> hd64(m, c->diag64_of(0));
            std::vector<T *> hdt(m, (T *)diagT(0));
            c->h2d(p_diag64, hd64.data(), m);
            c->h2d(p_diag, hdt.data(), m);
        }
        c->sync();
    }

    // room for `need` columns of V: grows by doubling up to r_max, keeping the
    // first r columns (device memory follows the rank, not r_max)
    void ensure_vcap(int need) {
        if (need <= vcap) return;
        if (need > rmax) throw Error{RCG_ERR_RANK_CAP, "basis V would exceed r_max columns"};
        const int nc = std::min(rmax, std::max(need, 2 * vcap));
        T *nv = c->alloc<T>((size_t)nc * ld);
        if (r > 0) RCG_CUDA_TRY(cudaMemcpyAsync(nv, V, sizeof(T) * (size_t)r * ld, cudaMemcpyDeviceToDevice, st));
        c->sync();
        c->release(V);
        V = nv;
        vcap = nc;
    }

    void ensure_ptr(int k) {
        if (k <= ptr_cap) return;
        c->release(d_ptrA); c->release(d_ptrB); c->release(d_ptrC);
        ptr_cap = std::max(k, 64);
        d_ptrA = (const void **)c->alloc<void *>(ptr_cap);
        d_ptrB = (const void **)c->alloc<void *>(ptr_cap);
        d_ptrC = (const void **)c->alloc<void *>(ptr_cap);
    }

    void ensure_append(int a) {
        if (a <= acap) return;
        for (void *p : std::vector<void *>{Wb, Qb, Cb, M, S, R, RK, Ri, Rhat, xn2, ratio_d, kept_d, d_K, d_cand})
            c->release(p);
        acap = std::max(a, 16);
        Wb = c->alloc<T>((size_t)acap * ld);
        Qb = c->alloc<T>((size_t)acap * ld);
        Cb = c->alloc<double>((size_t)(rmax + acap) * acap);
        M = c->alloc<double>((size_t)acap * acap);
        S = c->alloc<double>((size_t)acap * acap);
        R = c->alloc<double>((size_t)acap * acap);
        RK = c->alloc<double>((size_t)acap * acap);
        Ri = c->alloc<double>((size_t)acap * acap);
        Rhat = c->alloc<double>((size_t)acap * acap);
        xn2 = c->alloc<double>(acap);
        ratio_d = c->alloc<double>(acap);
        kept_d = c->alloc<int>(acap);
        d_K = c->alloc<int>(acap);
        d_cand = c->alloc<int>(acap);
    }

    void check_info(const char *what) {
        int info[2] = {0, 0};
        c->d2h(info, d_info, 2);
        c->sync();
        if (info[1] != 0) throw Error{RCG_ERR_TIMEOUT, "tensor-core product: an mbarrier wait ran out"};
        if (info[0] != 0) throw Error{RCG_ERR_NOT_SPD, std::string(what) + ": float64 Cholesky found a non-positive pivot"};
    }

    // C (ka x kb, ld ldc) = A^T B for n-long columns of stride ld.  float32
    // operands of at least 16 columns each go to the tensor cores (3xTF32,
    // float64 sum of the slices); the rest, and the float64 path, to the
    // CUDA-core kernels.  sym: A == B, ka == kb (upper tiles, mirrored).
    void prod_tn(const T *A, int ka, const T *B, int kb, double *C, int ldc, bool sym = false) {
        if constexpr (sizeof(T) == 4) {
            if (ka >= 16 && kb >= 16 && tc_gemm_tn_ok(ld, ld, A, B)) {
                const long long need = tc_gemm_tn_scratch(n, ka, kb, sym, nullptr, nullptr);
                if (need > tc_cap) {
                    c->release(tc_scr);
                    tc_cap = std::max(need, 2 * tc_cap);
                    tc_scr = c->alloc<float>((size_t)tc_cap);
                }
                tc_gemm_tn(st, n, A, ld, ka, B, ld, kb, C, ldc, false, sym, tc_scr, d_info + 1);
                return;
            }
        }
        gemm_tn<T, T>(st, n, A, ld, ka, B, ld, kb, C, ldc, false);
    }

    // A~_s applied to `cnt` columns (pointer lists on the host).
    void apply_cols(const std::vector<const T *> &src, const std::vector<T *> &dst, const std::vector<int> &samp) {
        const int cnt = (int)src.size();
        if (!cnt) return;
        ensure_ptr(cnt);
        std::vector<const void *> hs(cnt), hd(cnt), hg(cnt);
        for (int i = 0; i < cnt; ++i) { hs[i] = src[i]; hd[i] = dst[i]; hg[i] = diagT(samp[i]); }
        c->h2d(d_ptrA, hs.data(), cnt);
        c->h2d(d_ptrB, hd.data(), cnt);
        c->h2d(d_ptrC, hg.data(), cnt);
        apply_op<T>(st, g, D, (const T *const *)d_ptrC, (const T *const *)d_ptrA, (T *const *)d_ptrB, cnt, nullptr,
                    nullptr);
        // no synchronisation: the next call's copies into the pointer scratch
        // follow this kernel on the stream
    }

    struct Lane { int s, j; };          // a (sample, RHS) lane of a wave

    // ---- the paper's check and inner solver (float64 engine)
    // A~_s V = K R with R = R2 R1 (CholQR2): K in Kmr (ld), L_i = R_i^T in Lmr1/2
    double *Kmr = nullptr, *Kmr2 = nullptr, *Lmr1 = nullptr, *Lmr2 = nullptr, *Rmr = nullptr, *Rimr = nullptr;
    int kmr_cap = 0, mr_s = -1, mr_r = -1;
    void mr_factor(int s) {
        if constexpr (sizeof(T) == 8) {
            if (mr_s == s && mr_r == r) return;
            if (r > kmr_cap) {
                for (void *p : std::vector<void *>{Kmr, Kmr2, Lmr1, Lmr2, Rmr, Rimr}) c->release(p);
                kmr_cap = std::max(r, std::min(rmax, 2 * kmr_cap));
                Kmr = c->alloc<double>((size_t)kmr_cap * ld);
                Kmr2 = c->alloc<double>((size_t)kmr_cap * ld);
                for (double **p : {&Lmr1, &Lmr2, &Rmr, &Rimr}) *p = c->alloc<double>((size_t)kmr_cap * kmr_cap);
            }
            apply_cols64((const double *)V, Kmr, r, s);
            double *Ls[2] = {Lmr1, Lmr2};
            for (int pass = 0; pass < 2; ++pass) {
                gemm_tn<double, double>(st, n, Kmr, ld, r, Kmr, ld, r, Ls[pass], r, false);
                RCG_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), st));
                chol_inplace(st, Ls[pass], r, r, d_info);
                check_info("minimum-residual check: Cholesky QR of A V");
                lower_to_upper(st, Ls[pass], r, r, Rmr);
                tri_upper_inverse(st, Rmr, r, r, Rimr);
                gemm_nn<double, double>(st, n, Kmr, ld, r, Rimr, r, r, Kmr2, ld, 1.0, 0.0);
                std::swap(Kmr, Kmr2);
            }
            mr_s = s;
            mr_r = r;
        } else {
            (void)s;
            throw Error{RCG_ERR_INVALID, "the minimum-residual check runs in the float64 engine"};
        }
    }
    // recycled MINRES lanes: scalars [m][MR_NSC], dots, mu, alpha, step flags, 3 extra columns per lane
    double *mr_sc = nullptr, *mr_hd = nullptr, *mr_mu = nullptr, *mr_alpha = nullptr, *mr_ext = nullptr;
    int *mr_step = nullptr;
    int mr_cap = 0;
    void ensure_mres(int m) {
        if (m <= mr_cap) return;
        for (void *p : std::vector<void *>{mr_sc, mr_hd, mr_mu, mr_alpha, mr_ext, mr_step}) c->release(p);
        mr_cap = m;
        mr_sc = c->alloc<double>((size_t)m * MR_NSC);
        mr_hd = c->alloc<double>((size_t)m * KMAX);
        mr_mu = c->alloc<double>((size_t)m * KMAX);
        mr_alpha = c->alloc<double>(m);
        mr_step = c->alloc<int>(m);
        mr_ext = c->alloc<double>((size_t)m * 3 * ld);
    }
    // per-RHS recycling (the Sec. 6.3 comparison): new directions of RHS j in
    // a ring of KP_MAX columns, list entries -(2 + slot)
    T *Ppr = nullptr;
    std::vector<int> ppr_next;
    // The new direction of each listed lane, orthogonalised against its
    // recycle space (two Gram-Schmidt passes with the Euclidean Gram W^T W of
    // the lane's columns), normalised into the RHS's ring slot and appended to
    // its list: the columns of U_j stay well conditioned, which the projector
    // through H = (A~U_j)^T A~U_j needs.  kept[l] = 1 for the lanes stored.
    void per_rhs_store(const std::vector<int> &sel, const std::vector<Lane> &lanes, const LaneGeom &gm,
                       double tau, std::vector<int> &kept) {
        const int m = (int)sel.size();
        kept.assign(m, 0);
        if (std::find(sel.begin(), sel.end(), 1) == sel.end()) return;
        if constexpr (sizeof(T) == 8) {
            const int nrhs = c->nrhs;
            if (!Ppr) {
                Ppr = c->alloc<T>((size_t)nrhs * KP_MAX * ld);
                ppr_next.assign(nrhs, 0);
            }
            c->h2d(d_mask, sel.data(), m);
            mres_gram(st, n, gm, ls, d_mask, ls.gw, true);
            RCG_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), st));
            lane_inverse(st, ls.gw, ls.kdef, m, d_info);
            check_info("per-RHS recycle space Gram W^T W");
            double *w = (double *)qv;
            for (int pass = 0; pass < 2; ++pass) {
                const double *src = pass == 0 ? x64 : w;
                mres_dots(st, n, gm, ls, d_mask, src, mr_hd, true);
                mres_mu(st, ls, d_mask, mr_hd, mr_mu, mr_sc);
                mres_sub(st, n, gm, ls, d_mask, src, mr_mu, w, mr_sc);
            }
            std::vector<int> lst;
            for (int l = 0; l < m; ++l)
                if (sel[l]) lst.push_back(l);
            ensure_append((int)lst.size());
            c->h2d(d_cand, lst.data(), lst.size());
            norm2_lanes(st, n, (const double *const *)p_x64, d_cand, (int)lst.size(), xn2);
            std::vector<double> sch((size_t)m * MR_NSC), xh(lst.size());
            c->d2h(sch.data(), mr_sc, sch.size());
            c->d2h(xh.data(), xn2, xh.size());
            c->sync();
            for (size_t i = 0; i < lst.size(); ++i) {
                const int l = lst[i], j = lanes[l].j;
                const double wn2 = sch[(size_t)l * MR_NSC + MR_XI2];
                if (!(std::sqrt(wn2) > tau * std::sqrt(xh[i]))) continue;     // nothing new for U_j
                const int slot = ppr_next[j];
                ppr_next[j] = (slot + 1) % KP_MAX;
                auto &pl = priv[j];
                pl.erase(std::remove(pl.begin(), pl.end(), -(2 + slot)), pl.end());   // the slot's old direction
                T *dst = Ppr + ((long long)j * KP_MAX + slot) * ld;
                k_scaled_copy<T><<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(
                    n, w + (long long)l * ld, mr_sc + (size_t)l * MR_NSC + MR_XI2, dst);
                ++c->launches;
                RCG_CHECK_LAUNCH();
                pl.push_back(-(2 + slot));
                while (k_u + (int)pl.size() > std::min(c->opt.k_cap, k_u + KP_MAX) && !pl.empty()) pl.erase(pl.begin());
                kept[l] = 1;
            }
            c->sync();
        } else {
            (void)lanes; (void)gm; (void)tau;
            throw Error{RCG_ERR_INVALID, "per-RHS recycling runs in the float64 engine"};
        }
    }

    // float64 scratch for the new basis columns and their images
    double *Q64 = nullptr, *AQ64 = nullptr;
    int aq64_cap = 0;
    void ensure_aq64(int a) {
        if (a <= aq64_cap) return;
        c->release(Q64); c->release(AQ64);
        aq64_cap = std::max(a, 16);
        Q64 = c->alloc<double>((size_t)aq64_cap * ld);
        AQ64 = c->alloc<double>((size_t)aq64_cap * ld);
    }
    // float64 A~_s applied to cnt contiguous float64 columns
    void apply_cols64(const double *src, double *dst, int cnt, int s) {
        ensure_ptr(cnt);
        std::vector<const void *> hs(cnt), hd(cnt), hg(cnt);
        for (int i = 0; i < cnt; ++i) {
            hs[i] = src + (long long)i * ld;
            hd[i] = dst + (long long)i * ld;
            hg[i] = c->diag64_of(s);
        }
        c->h2d(d_ptrA, hs.data(), cnt);
        c->h2d(d_ptrB, hd.data(), cnt);
        c->h2d(d_ptrC, hg.data(), cnt);
        apply_op<double>(st, g, c->D64, (const double *const *)d_ptrC, (const double *const *)d_ptrA,
                         (double *const *)d_ptrB, cnt, nullptr, nullptr);
    }

    // Out = V Y (+ beta Out) with float64 accuracy: V is float64 in RCG_FP64; in
    // RCG_MIXED the float32 basis is lifted with double-float accumulation.
    void lift(const T *Vb, int k, const double *Y, int ldy, int m, double *Out, long long ldo, double beta) {
        if (mixed)
            gemm_nn_df(st, n, (const float *)Vb, ld, k, Y, ldy, m, Out, ldo, beta);
        else
            gemm_nn<T, double>(st, n, Vb, ld, k, Y, ldy, m, Out, ldo, 1.0, beta);
    }

    // ----------------------------------------------------- Galerkin matrices
    double *delta_weights(int s) {
        if (!dw[s]) dw[s] = c->alloc<double>(ld);
        if (dw_star[s] != s_star) {
            scaled_diff(st, n, c->mu64 + (long long)s * ld, c->mu64 + (long long)s_star * ld, c->h * c->h, dw[s]);
            if (mixed) {
                if (!dwl[s]) dwl[s] = c->alloc<int>((size_t)(n + 31) / 32);
                tc_block_list(st, n, dw[s], dwl[s], dwc + s);
            }
            dw_star[s] = s_star;
        }
        return dw[s];
    }

    // Out (n x m) = alpha A C + beta Out with A (n x k, stride ld) and C (k x m,
    // float64): tensor cores for float32 with k, m >= 16, CUDA cores otherwise.
    void prod_nn(const T *A, int k, const double *C, int ldc, int m, T *Out, double alpha, double beta) {
        if constexpr (sizeof(T) == 4) {
            if (k >= 16 && m >= 16 && ld % 4 == 0 && ((uintptr_t)A & 15) == 0) {
                const long long need = tc_gemm_nn_scratch(k, m);
                if (need > tc_cap) {
                    c->release(tc_scr);
                    tc_cap = std::max(need, 2 * tc_cap);
                    tc_scr = c->alloc<float>((size_t)tc_cap);
                }
                tc_gemm_nn(st, n, A, ld, k, C, ldc, m, Out, ld, alpha, beta, tc_scr, d_info + 1);
                return;
            }
        }
        gemm_nn<T, T>(st, n, A, ld, k, C, ldc, m, Out, ld, alpha, beta);
    }

    // C (ka x ka, ld ldc) += A^T diag(w) A: the weighted Gram of the check and the
    // reduced model; tensor cores (only the 32-row blocks in blist) for float32.
    void gram_w_acc(const T *A, int ka, double *C, int ldc, const double *w, const int *blist, const int *bcount) {
        if constexpr (sizeof(T) == 4) {
            if (ka >= 16 && blist && tc_gemm_tn_ok(ld, ld, A, A)) {
                const long long need = tc_gemm_tn_scratch(n, ka, ka, true, nullptr, nullptr);
                if (need > tc_cap) {
                    c->release(tc_scr);
                    tc_cap = std::max(need, 2 * tc_cap);
                    tc_scr = c->alloc<float>((size_t)tc_cap);
                }
                tc_gemm_tn(st, n, A, ld, ka, A, ld, ka, C, ldc, true, true, tc_scr, d_info + 1, w, blist, bcount);
                return;
            }
        }
        gemm_tn_acc<T, T, double>(st, n, A, ld, ka, A, ld, ka, C, ldc, true, w);
    }

    // ---- diffusion tracking the absorption: operator differences and derivatives
    // (dg diagonal, dw face weights towards +x, +y, +z) and products over their rows
    double *tk_dg = nullptr, *tk_dw = nullptr, *tk_touch = nullptr;
    int *tk_bl = nullptr, *tk_bc = nullptr;
    T *tk_Xc = nullptr;
    double *tk_Yc = nullptr;
    long long tk_cap = 0;
    // the point of a reduced-model evaluation: D, face weights, diagonal, weights
    double *tp_D = nullptr, *tp_W = nullptr, *tp_diag = nullptr, *tp_w = nullptr, *tp_G = nullptr, *tp_P = nullptr;
    double *tp_dwt = nullptr;
    int tp_dwt_cap = 0;
    void ensure_track() {
        if (tk_dg) return;
        tk_dg = c->alloc<double>(ld);
        tk_dw = c->alloc<double>((size_t)3 * ld);
        tk_touch = c->alloc<double>(ld);
        tk_bl = c->alloc<int>((size_t)(n + 31) / 32);
        tk_bc = c->alloc<int>(1);
    }
    // G (ka x ka, ld ldg) += X^T dA X with dA the operator difference or
    // derivative in (tk_dg, tk_dw): Y = dA X in float64 on the 32-row blocks
    // where dA has a nonzero row, next to those rows of X, then one product
    // per chunk of blocks (double-float for a float32 X, float64 otherwise).
    void delta_gram(const T *X, int ka, double *G, int ldg) {
        if (ka <= 0) return;
        track_touch(st, g, tk_dg, tk_dw, tk_touch);
        tc_block_list(st, n, tk_touch, tk_bl, tk_bc);
        int nb = 0;
        c->d2h(&nb, tk_bc, 1);
        c->sync();
        if (nb <= 0) return;
        const long long max_blocks = std::max<long long>(1, (1LL << 27) / ((long long)ka * 32));   // ~1 GiB of Y
        const int bchunk = (int)std::min<long long>(nb, max_blocks);
        const long long need = (long long)bchunk * 32 * ka;
        if (need > tk_cap) {
            c->release(tk_Xc);
            c->release(tk_Yc);
            tk_cap = need;
            tk_Xc = c->alloc<T>((size_t)need);
            tk_Yc = c->alloc<double>((size_t)need);
        }
        for (int b0 = 0; b0 < nb; b0 += bchunk) {
            const int nbc = std::min(bchunk, nb - b0);
            const long long rows = (long long)nbc * 32;
            delta_rows<T>(st, g, tk_bl, b0, nbc, tk_dg, tk_dw, X, ld, ka, tk_Xc, tk_Yc, rows);
            if constexpr (sizeof(T) == 4)
                gemm_tn_df(st, rows, (const float *)tk_Xc, rows, ka, tk_Yc, rows, ka, G, ldg, true);
            else
                gemm_tn<double, double>(st, rows, (const double *)tk_Xc, rows, ka, tk_Yc, rows, ka, G, ldg, true);
        }
    }

    // G = C_* + V^T (A~_s - A~_*) V (r x r) and its Cholesky factor L: with a fixed
    // D the difference is diag(h^2 (mu_s - mu_*)); with D tracking mu it also
    // changes every face weight on and around the support of mu_s - mu_*.
    void galerkin(int s, double *G, double *L, bool reset_info = true) {
        RCG_CUDA_TRY(cudaMemcpy2DAsync(G, sizeof(double) * rmax, Cstar, sizeof(double) * rmax, sizeof(double) * r, r,
                                       cudaMemcpyDeviceToDevice, st));
        if (s != s_star && c->track()) {
            ensure_track();
            scaled_diff(st, n, c->diag64_of(s), c->diag64_of(s_star), 1.0, tk_dg);
            scaled_diff(st, 3 * ld, c->Ws64_of(s), c->Ws64_of(s_star), 1.0, tk_dw);
            delta_gram(V, r, G, rmax);
        } else if (s != s_star) {
            const double *w = delta_weights(s);
            gram_w_acc(V, r, G, rmax, w, mixed ? dwl[s] : nullptr, mixed ? dwc + s : nullptr);
        }
        RCG_CUDA_TRY(cudaMemcpy2DAsync(L, sizeof(double) * rmax, G, sizeof(double) * rmax, sizeof(double) * r, r,
                                       cudaMemcpyDeviceToDevice, st));
        if (reset_info) RCG_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), st));
        chol_inplace(st, L, rmax, r, d_info);
    }

    // check: false leaves the factorisation's status in d_info for one
    // check_info after several samples (the wave order)
    std::pair<double *, double *> galerkin_for(int s, bool seq, bool check = true) {
        if (seq) {
            if (gs_sample != s || gs_r != r) {
                galerkin(s, Gs, Ls);
                check_info("Galerkin matrix V^T A V");
                gs_sample = s;
                gs_r = r;
            }
            return {Gs, Ls};
        }
        if (!Gw[s]) { Gw[s] = c->alloc<double>((size_t)rmax * rmax); Lw[s] = c->alloc<double>((size_t)rmax * rmax); }
        galerkin(s, Gw[s], Lw[s], check);
        if (check) check_info("Galerkin matrix V^T A V");
        return {Gw[s], Lw[s]};
    }

    // Cb (r+ak x ak) = [V Q]^T (A~_s Q) for the ak new columns Q = V(:, r..r+ak)
    // (the border of C_* or G_s), with A~_s Q in float64: double-float products
    // for the float32 basis, float64 otherwise.  In chunks of AQ_CHUNK columns,
    // so the float64 scratch stays small for a wave's large appends.
    static constexpr int AQ_CHUNK = 32;
    void border_cols(int ak, int s) {
        ensure_aq64(std::min(ak, AQ_CHUNK));
        for (int a0 = 0; a0 < ak; a0 += AQ_CHUNK) {
            const int na = std::min(AQ_CHUNK, ak - a0);
            convert_cols<T, double>(st, n, V + (long long)(r + a0) * ld, ld, Q64, ld, na);
            apply_cols64(Q64, AQ64, na, s);
            double *out = Cb + (long long)a0 * (r + ak);
            if constexpr (sizeof(T) == 4) gemm_tn_df(st, n, (const float *)V, ld, r + ak, AQ64, ld, na, out, r + ak, false);
            else gemm_tn<T, double>(st, n, V, ld, r + ak, AQ64, ld, na, out, r + ak, false);
        }
    }

    // ------------------------------------------------------------ append
    // Ordered rank-revealing append of the solutions in lanes `cand` (order
    // = priority).  Returns per-candidate kept flags and ratios.
    void append(const std::vector<int> &cand, double tau, int border_sample, std::vector<int> &kept,
                std::vector<double> &ratio) {
        const int a = (int)cand.size();
        kept.assign(a, 0);
        ratio.assign(a, 0.0);
        if (!a) return;
        ensure_append(a);
        c->h2d(d_cand, cand.data(), a);
        convert_lanes<double, T>(st, n, (const double *const *)p_x64, d_cand, a, Wb, ld);
        norm2_lanes(st, n, (const double *const *)p_x64, d_cand, a, xn2);
        for (int pass = 0; pass < 2 && r > 0; ++pass) {   // W <- (I - V V^T)^2 X
            prod_tn(V, r, Wb, a, Cb, r);
            prod_nn(V, r, Cb, r, a, Wb, -1.0, 1.0);
        }
        prod_tn(Wb, a, Wb, a, M, a, true);
        ordered_drop_chol(st, M, a, xn2, S, tau, R, kept_d, ratio_d);
        c->d2h(kept.data(), kept_d, a);
        c->d2h(ratio.data(), ratio_d, a);
        c->sync();
        std::vector<int> K;
        for (int i = 0; i < a; ++i)
            if (kept[i]) K.push_back(i);
        const int ak = (int)K.size();
        if (!ak) return;
        if (r + ak > rmax) throw Error{RCG_ERR_RANK_CAP, "basis V would exceed r_max columns"};
        c->h2d(d_K, K.data(), ak);
        // Q = W_K R_K^-1
        gather_sub(st, R, a, d_K, ak, RK);
        tri_upper_inverse(st, RK, ak, ak, Ri);
        scatter_rows(st, Ri, ak, d_K, a, Rhat);
        prod_nn(Wb, a, Rhat, a, ak, Qb, 1.0, 0.0);
        // second pass: Q <- (I - V V^T) Q, then Q R2^-1 with R2^T R2 = Q^T Q
        if (r > 0) {
            prod_tn(V, r, Qb, ak, Cb, r);
            prod_nn(V, r, Cb, r, ak, Qb, -1.0, 1.0);
        }
        prod_tn(Qb, ak, Qb, ak, M, ak, true);
        RCG_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), st));
        chol_inplace(st, M, ak, ak, d_info);
        check_info("append second pass Q^T Q");
        lower_to_upper(st, M, ak, ak, RK);
        tri_upper_inverse(st, RK, ak, ak, Ri);
        ensure_vcap(r + ak);
        prod_nn(Qb, ak, Ri, ak, ak, V + (long long)r * ld, 1.0, 0.0);
        // C_* bordered with [V Q]^T A~_* Q.  The stencil and the products are
        // float64 in both modes: for smooth columns A~ Q cancels to ~lambda_min
        // |Q|, so a float32 stencil would lose 3 digits of the Galerkin matrix
        // that the check, the deflation matrices and the reduced model solve with.
        border_cols(ak, s_star);
        border_write(st, Cstar, rmax, r, ak, Cb, r + ak);
        if (border_sample >= 0 && gs_sample == border_sample && gs_r == r) {
            border_cols(ak, border_sample);
            border_write(st, Gs, rmax, r, ak, Cb, r + ak);
            copy_new_rows(st, Gs, Ls, rmax, r, ak);
            RCG_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), st));
            chol_border(st, Ls, rmax, r, ak, d_info);
            check_info("bordered Galerkin factor");
            gs_r = r + ak;
        }
        r += ak;
    }

    // -------------------------------------------------------------- wave

    void wave(const std::vector<Lane> &lanes, bool seed_mode, bool seq, std::vector<rcg_stat> &out) {
        const int m = (int)lanes.size();
        ensure_lanes(m);
        const double tau = seed_mode ? c->opt.tau_rank : c->opt.tau_rank;
        // the paper's own check and inner solver (float64 engine), and per-RHS recycling only
        const bool use_mres = !mixed && c->opt.inner == RCG_MINRES;
        const bool mr_check = !mixed && c->opt.check == RCG_MR && !seed_mode;
        const bool per_rhs = c->opt.recycle == RCG_PER_RHS && !seed_mode;
        std::vector<int> lnode(m), samp(m);
        std::vector<double> lw(m), ltol(m);
        std::vector<double *> hdiag64(m);
        std::vector<T *> hdiag(m);
        for (int l = 0; l < m; ++l) {
            lnode[l] = c->rhs_node[lanes[l].j];
            lw[l] = c->rhs_w[lanes[l].j];
            ltol[l] = c->tol[lanes[l].j];
            samp[l] = lanes[l].s;
            hdiag64[l] = c->diag64_of(lanes[l].s);
            hdiag[l] = (T *)diagT(lanes[l].s);
        }
        c->h2d(d_lnode, lnode.data(), m);
        c->h2d(d_lw, lw.data(), m);
        c->h2d(p_diag64, hdiag64.data(), m);
        c->h2d(p_diag, hdiag.data(), m);
        out.assign(m, rcg_stat{});
        for (int l = 0; l < m; ++l) { out[l].sample = lanes[l].s; out[l].rhs = lanes[l].j; }

        // ---- check: Galerkin guess from range(V) and its float64 residual
        cudaEvent_t e0, e1, e2, e3;
        RCG_CUDA_TRY(cudaEventCreate(&e0)); RCG_CUDA_TRY(cudaEventCreate(&e1));
        RCG_CUDA_TRY(cudaEventCreate(&e2)); RCG_CUDA_TRY(cudaEventCreate(&e3));
        RCG_CUDA_TRY(cudaEventRecord(e0, st));
        std::vector<int> grp_begin;        // lanes sorted by sample: group starts
        for (int l = 0; l < m; ++l)
            if (l == 0 || samp[l] != samp[l - 1]) grp_begin.push_back(l);
        grp_begin.push_back(m);
        std::map<int, std::pair<double *, double *>> gal;
        const bool need_gal = !((c->opt.check == RCG_MR || c->opt.recycle == RCG_PER_RHS) && !seed_mode &&
                                c->opt.inner == RCG_MINRES && !mixed);
        if (r > 0 && need_gal) {
            // wave order: all samples' matrices and factors, then one status check
            if (!seq) RCG_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), st));
            for (size_t gi = 0; gi + 1 < grp_begin.size(); ++gi) {
                const int s = samp[grp_begin[gi]];
                if (!gal.count(s)) gal[s] = galerkin_for(s, seq, seq);
            }
            if (!seq) check_info("Galerkin matrix V^T A V");
        }
        const T *Vc = V;
        auto project = [&](bool first) {
            // Yb = V^T b (first) or V^T r; Y = G^-1 Yb; x64 (+)= V Y
            if (first) gather_rows<T>(st, Vc, ld, r, d_lnode, d_lw, m, Yb, rmax);
            else prod_tn(Vc, r, rv, m, Yb, rmax);
            for (size_t gi = 0; gi + 1 < grp_begin.size(); ++gi) {
                const int l0 = grp_begin[gi], l1 = grp_begin[gi + 1];
                double *L = gal[samp[l0]].second;
                trsv_lower_batched(st, L, rmax, r, Yb + (long long)l0 * rmax, rmax, l1 - l0, false);
                trsv_lower_batched(st, L, rmax, r, Yb + (long long)l0 * rmax, rmax, l1 - l0, true);
            }
            lift(Vc, r, Yb, rmax, m, x64, ld, first ? 0.0 : 1.0);
        };
        // nact: how many lanes the mask selects (sizes the grid for them)
        auto residual = [&](std::vector<double> &rr_h, const int *mask, int nact = -1) {
            RCG_CUDA_TRY(cudaMemsetAsync(d_rr, 0, sizeof(double) * m, st));
            residual64(st, g, c->W64, (const double *const *)p_diag64, (const double *const *)p_x64,
                       mixed ? nullptr : (double *const *)p_r, mixed ? (float *const *)p_r : nullptr, m, d_lnode, d_lw,
                       d_rr, mask, nact < 0 ? m : nact);
            rr_h.resize(m);
            c->d2h(rr_h.data(), d_rr, m);
            c->sync();
        };
        // the minimum-residual guess from range(V): c = K^T b (a row of K), y = R^-1 c
        // with A~_s V = K R2 R1 (CholQR, two passes), x0 = V y
        auto mr_project = [&]() {
            for (size_t gi = 0; gi + 1 < grp_begin.size(); ++gi) {
                const int l0 = grp_begin[gi], l1 = grp_begin[gi + 1];
                mr_factor(samp[l0]);
                gather_rows<double>(st, (const double *)Kmr, ld, r, d_lnode + l0, d_lw + l0, l1 - l0,
                                    Yb + (long long)l0 * rmax, rmax);
                trsv_lower_batched(st, Lmr2, r, r, Yb + (long long)l0 * rmax, rmax, l1 - l0, true);
                trsv_lower_batched(st, Lmr1, r, r, Yb + (long long)l0 * rmax, rmax, l1 - l0, true);
            }
            lift(V, r, Yb, rmax, m, x64, ld, 0.0);
        };
        if (r > 0 && !per_rhs) {
            if (mr_check) mr_project();
            else project(true);
        } else {
            for (int l = 0; l < m; ++l) RCG_CUDA_TRY(cudaMemsetAsync(x64 + (long long)l * ld, 0, sizeof(double) * n, st));
        }
        std::vector<double> rr_h;
        residual(rr_h, nullptr);
        if (r > 0 && !seed_mode && !mr_check && !per_rhs) {
            for (int step = 0; step < c->opt.check_refine; ++step) {
                project(false);
                residual(rr_h, nullptr);
            }
        }
        std::vector<double> relres0(m);
        for (int l = 0; l < m; ++l) relres0[l] = std::sqrt(rr_h[l]) / std::fabs(lw[l]);
        RCG_CUDA_TRY(cudaEventRecord(e1, st));

        // ---- deflated CG on the lanes the check rejected
        std::vector<int> act(m, 0), done(m, 0), restarts(m, 0), status(m, RCG_OK);
        std::vector<double> relres(relres0);
        int nact = 0;
        for (int l = 0; l < m; ++l) {
            out[l].relres0 = relres0[l];
            if (relres0[l] > ltol[l] || seed_mode) {
                if (relres0[l] > ltol[l]) { act[l] = 1; ++nact; }
            }
        }
        std::vector<int> iters_h(m, 0);
        std::vector<int> prh_kept;          // per-RHS recycling: lanes whose new direction joined U_j
        // learned augmentation (float32 engine): features of the check residuals,
        // the network's coarse prediction, coarse x0 when recording pairs
        Cnn *net = nullptr;
        if constexpr (sizeof(T) == 4) {
            if (!seed_mode && c->cnn && (c->cnn->record || (c->opt.learned && c->cnn->have))) net = c->cnn.get();
        }
        const bool use_aug = net && c->opt.learned && net->have;
        bool drop_first = false;       // RCG_LEARN_START: the first start drops the learned columns
        std::vector<int> alanes;
        if (net && nact) {
            for (int l = 0; l < m; ++l)
                if (act[l]) alanes.push_back(l);
            const int na = (int)alanes.size();
            const long long Vc = net->geom.V;
            ensure_learn(m);
            std::vector<const float *> hr(na);
            std::vector<const double *> hm(na), hx(na);
            for (int a = 0; a < na; ++a) {
                const int l = alanes[a];
                hr[a] = (const float *)(rv + (long long)l * ld);
                hm[a] = c->mu64 + (long long)samp[l] * ld;
                hx[a] = x64 + (long long)l * ld;
            }
            c->h2d(d_lr, hr.data(), na);
            c->h2d(d_lm, hm.data(), na);
            c->h2d(d_lx, hx.data(), na);
            net->ensure(net->feat, net->feat_cap, (long long)na * 2 * Vc);
            net->features(st, d_lr, d_lm, na, net->feat);
            if (net->record) {
                net->ensure(net->x0c, net->x0c_cap, (long long)na * Vc);
                net->pool64(st, d_lx, net->x0c, na, -1.f, false);
            }
            if (use_aug) {
                net->ensure(net->outc, net->outc_cap, (long long)na * Vc);
                net->forward(st, net->feat, na, net->outc);
            }
        }
        if (nact) {
            // deflation spaces: U_j = [V(:, 0:k_u), X_0(:, j), V(:, priv_j)] (seed: V(:, 0:k_u))
            std::vector<int> spec((size_t)m * KMAX, 0), kdef(m, 0), kp(m, 0), si(m, 0);
            std::vector<double *> sxp(m, nullptr), gsl(m, nullptr);
            std::vector<int> samples_in;
            for (int l = 0; l < m; ++l)
                if (act[l] && std::find(samples_in.begin(), samples_in.end(), samp[l]) == samples_in.end())
                    samples_in.push_back(samp[l]);
            const int ku = std::min(k_u, r);
            // A~_s U_0 per sample: the first k_u basis columns never change after
            // the seed, so the images are cached per sample slot
            if (samples_in != au0_samples || ku != au0_ku || au0_star != s_star) {
                if ((int)samples_in.size() * ku > au0_cap) {
                    c->release(au0);
                    au0_cap = (int)samples_in.size() * ku;
                    au0 = c->alloc<T>((size_t)std::max(au0_cap, 1) * ld);
                }
                au0_valid = false;
            }
            std::vector<const T *> asrc;
            std::vector<T *> adst;
            std::vector<int> asamp;
            if (!au0_valid) {
                for (size_t s2 = 0; s2 < samples_in.size(); ++s2)
                    for (int q = 0; q < ku; ++q) {
                        asrc.push_back(V + (long long)q * ld);
                        adst.push_back(au0 + ((long long)s2 * ku + q) * ld);
                        asamp.push_back(samples_in[s2]);
                    }
                au0_samples = samples_in;
                au0_ku = ku;
                au0_star = s_star;
                au0_valid = true;
            }
            int kmax_used = 0, kp_max = 0;
            for (int l = 0; l < m; ++l) {
                if (!act[l]) continue;
                std::vector<int> sp;
                for (int q = 0; q < ku; ++q) sp.push_back(q);
                if (!seed_mode)
                    for (int e : priv[lanes[l].j]) sp.push_back(e);
                if ((int)sp.size() - ku > KP_MAX) sp.erase(sp.begin() + ku, sp.begin() + ((int)sp.size() - KP_MAX));
                kdef[l] = (int)sp.size();
                kp[l] = kdef[l] - ku;
                kp_max = std::max(kp_max, kp[l]);
                kmax_used = std::max(kmax_used, kdef[l]);
                si[l] = (int)(std::find(samples_in.begin(), samples_in.end(), samp[l]) - samples_in.begin());
                for (int q = 0; q < (int)sp.size(); ++q) spec[(size_t)l * KMAX + q] = sp[q];
                sxp[l] = sX0 ? sX0 + (long long)lanes[l].j * rmax : nullptr;
                gsl[l] = gal.count(samp[l]) ? gal[samp[l]].first : nullptr;
            }
            // one more private slot for the network's column where it fits
            std::vector<int> aug(m, 0);
            int kps = kp_max;
            if (use_aug)
                for (int l = 0; l < m; ++l) {
                    aug[l] = act[l] && kp[l] < KP_MAX;
                    kps = std::max(kps, kp[l] + aug[l]);
                }
            const long long npriv = (long long)m * kps;
            if (npriv > awp_cap) {
                c->release(awp);
                awp_cap = npriv;
                awp = c->alloc<T>((size_t)npriv * ld);
            }
            // private W columns by address (V, X_0, or the network's column),
            // their images A~_s W next to each other per lane
            std::vector<const void *> hwpp((size_t)m * KPT, (const void *)V);
            for (int l = 0; l < m; ++l)
                for (int q = 0; q < kp[l]; ++q) {
                    const int e = spec[(size_t)l * KMAX + ku + q];
                    const T *w = e >= 0 ? V + (long long)e * ld
                                 : e == -1 ? X0 + (long long)lanes[l].j * ld
                                           : Ppr + ((long long)lanes[l].j * KP_MAX + (-e - 2)) * ld;
                    hwpp[(size_t)l * KPT + q] = w;
                    asrc.push_back(w);
                    adst.push_back(awp + ((long long)l * kps + q) * ld);
                    asamp.push_back(samp[l]);
                }
            // the network's column x_hat in slot kp[l] of the lane, then A~ x_hat with the others
            std::vector<int> aug_l;
            if (use_aug) {
                std::vector<float *> hd;
                std::vector<int> rows;
                int naug = 0;
                for (size_t a = 0; a < alanes.size(); ++a) naug += aug[alanes[a]];
                if (naug > xhb_cap) {
                    c->release(xhb);
                    xhb_cap = naug;
                    xhb = c->alloc<T>((size_t)naug * ld);
                }
                for (size_t a = 0; a < alanes.size(); ++a) {
                    const int l = alanes[a];
                    if (!aug[l]) continue;
                    T *w = xhb + (long long)hd.size() * ld;
                    hwpp[(size_t)l * KPT + kp[l]] = w;
                    hd.push_back((float *)w);
                    rows.push_back((int)a);
                    aug_l.push_back(l);
                    asrc.push_back(w);
                    adst.push_back(awp + ((long long)l * kps + kp[l]) * ld);
                    asamp.push_back(samp[l]);
                }
                if (!hd.empty()) {
                    c->h2d(d_ldst, hd.data(), hd.size());
                    c->h2d(d_arow, rows.data(), rows.size());
                    net->upsample(st, net->outc, d_ldst, d_arow, (int)hd.size());
                }
            }
            c->h2d(d_wpp, hwpp.data(), hwpp.size());
            apply_cols(asrc, adst, asamp);
            c->h2d(d_spec, spec.data(), (size_t)m * KMAX);
            c->h2d(ls.kdef, kdef.data(), m);
            c->h2d(d_si, si.data(), m);
            c->h2d(d_kp, kp.data(), m);
            c->h2d(d_sx, sxp.data(), m);
            c->h2d(d_gsl, gsl.data(), m);
            LaneGeom gm{};
            gm.ld = ld;
            gm.k_u = ku;
            gm.kp_max = std::max(kps, 1);
            gm.kp_sel = gm.kp_max;
            gm.x = xc; gm.r = rv; gm.p = pv; gm.q = qv;
            gm.wu = V; gm.awu = au0; gm.awp = awp; gm.wpp = d_wpp;
            gm.si = d_si; gm.kp = d_kp;
            ls.nl = m;                     // the kernels of this wave launch over its m lanes
            if (kmax_used > 0) {
                if (use_mres) {
                    // recycled MINRES: H = (A~ U_j)^T A~ U_j, whose inverse gives the
                    // projector away from range(A~ U_j) = range(K_j)
                    c->h2d(d_mask, act.data(), m);
                    mres_gram(st, n, gm, ls, d_mask, ls.gw);
                } else {
                    lane_gw(st, (const double *const *)d_gsl, rmax, r, d_spec, (const double *const *)d_sx, ls.kdef,
                            ls.gw, m);
                }
                RCG_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), st));
                lane_inverse(st, ls.gw, ls.kdef, m, d_info);
                check_info(use_mres ? "recycle matrix (A U_j)^T A U_j" : "deflation matrix U_j^T A U_j");
            }
            if (!aug_l.empty()) {
                // Galerkin pivot of x_hat against U_j; kept columns border G_W^-1 on the device
                const int nq = (int)aug_l.size();
                c->h2d(d_aug_l, aug_l.data(), nq);
                aug_dots(st, n, ld, (const float *)V, ku, (const float *const *)d_wpp, (const float *)awp, kps, d_kp, d_aug_l, nq,
                         d_cd);
                aug_border(st, ls.gw, ls.kdef, d_kp, d_aug_l, nq, d_cd, c->opt.tau_rank, d_kept);
                std::vector<int> kh(nq);
                c->d2h(kh.data(), d_kept, nq);
                c->sync();
                for (int i = 0; i < nq; ++i) out[aug_l[i]].augmented = kh[i];
                if (c->opt.learned_mode == RCG_LEARN_START) {
                    // the kept columns serve the first projection only
                    std::vector<int> dm(m, 0);
                    for (int i = 0; i < nq; ++i) dm[aug_l[i]] = kh[i];
                    c->h2d(d_drop, dm.data(), m);
                    drop_first = true;
                }
            }
            // thresholds and the first (re)start
            std::vector<double> thr(m, 0.0);
            auto set_thresh = [&](int l, double rnorm) {
                const double target = ltol[l] * std::fabs(lw[l]);
                thr[l] = mixed ? std::max(0.5 * target, c->opt.inner_eta * rnorm) : target;
            };
            for (int l = 0; l < m; ++l)
                if (act[l]) set_thresh(l, std::sqrt(rr_h[l]));
            RCG_CUDA_TRY(cudaMemsetAsync(ls.iters, 0, sizeof(int) * ls.m, st));
            RCG_CUDA_TRY(cudaMemsetAsync(ls.active, 0, sizeof(int) * ls.m, st));
            RCG_CUDA_TRY(cudaMemsetAsync(ls.flag, 0, sizeof(int) * ls.m, st));
            RCG_CUDA_TRY(cudaMemsetAsync(ls.xt, 0xFF, sizeof(int) * ls.m, st));    // no pending x step
            RCG_CUDA_TRY(cudaMemsetAsync(d_mask, 0, sizeof(int) * ls.m, st));
            c->h2d(ls.thresh, thr.data(), m);
            c->h2d(d_mask, act.data(), m);
            ls.prof = c->ktimer.on ? c->d_prof : nullptr;
            int t = 0;

            std::vector<int> flag_h(m), active_h(m);
            // lanes selected by `sel` and tiles of <= 32 of them per sample slot
            const bool vec = mixed && cg4_supported(g) && !c->track();     // the float4 stencils take one fixed D
            // the scalar path replays a CUDA graph of a 6-iteration chunk: its ring
            // slots (t mod 3, t mod 2) repeat every 6 iterations and restarts fall
            // on chunk boundaries, so one capture per wave serves every chunk
            const bool graph = !vec && !c->ktimer.on;
            const int chunk = graph ? 6 : (m > 1 ? 8 : 12);
            CgGraph cgg(st);
            LaneList ll{d_alist, 0, d_tlane, d_tsi, d_tcnt, 0};
            if (mixed) {                   // the lanes' p columns and the sample diagonals (TMA stencil)
                ll.pbase = (const float *)pv;
                ll.pld = ld;
                ll.pcols = m;
                ll.gbase = c->diag32;
                ll.gslots = c->opt.max_samples;
            }
            auto build_list_of = [&](const std::vector<int> &sel) {
                std::vector<int> al, tl, tsi, tcnt;
                for (int l = 0; l < m; ++l)
                    if (sel[l]) al.push_back(l);
                for (size_t q = 0; q < al.size();) {
                    const int s0 = si[al[q]];
                    int cnt = 0;
                    const size_t base = tl.size();
                    tl.resize(base + 32, -1);
                    while (q < al.size() && cnt < 32 && si[al[q]] == s0) tl[base + cnt++] = al[q++];
                    tsi.push_back(s0);
                    tcnt.push_back(cnt);
                }
                ll.na = (int)al.size();
                ll.ntiles = (int)tcnt.size();
                if (ll.na) {
                    c->h2d(d_alist, al.data(), al.size());
                    c->h2d(d_tlane, tl.data(), tl.size());
                    c->h2d(d_tsi, tsi.data(), tsi.size());
                    c->h2d(d_tcnt, tcnt.data(), tcnt.size());
                }
            };
            auto build_list = [&]() {
                std::vector<int> sel(m, 0);
                for (int l = 0; l < m; ++l) sel[l] = act[l] && !done[l];
                build_list_of(sel);
            };
            // (re)start the lanes flagged in `mask_h` (also uploaded to d_mask);
            // the first start drops the learned columns after its projection
            // under RCG_LEARN_START
            auto restart = [&](const std::vector<int> &mask_h) {
                int *drop = drop_first ? d_drop : nullptr;
                drop_first = false;
                if (vec) {
                    lane_zero(st, ls, d_mask);
                    build_list_of(mask_h);
                    cg_restart4(st, g, gm, ls, ll, t, mu_f, beta_f, drop);
                } else {
                    cg_restart<T>(st, g, gm, ls, t, d_mask, drop);
                }
            };
            if (use_mres) {
                // recycled MINRES cycles (minres.cu) until the float64 residual meets tol
                ensure_mres(ls.m);              // the kernels clear per-lane arrays over the capacity
                ls.maxit = c->opt.maxit;
                std::vector<double> sch((size_t)m * MR_NSC, 0.0);
                for (int l = 0; l < m; ++l) sch[(size_t)l * MR_NSC + MR_THRESH] = thr[l];
                c->h2d(mr_sc, sch.data(), sch.size());
                LaneGeom gq = gm;
                gq.r = gm.q;                               // (A~W)^T of A~ y at the end of a cycle
                auto cycle_start = [&](const std::vector<int> &mask_h) {
                    c->h2d(d_mask, mask_h.data(), m);
                    mres_dots(st, n, gm, ls, d_mask, (const double *)gm.r, mr_hd);
                    mres_mu(st, ls, d_mask, mr_hd, mr_mu, mr_sc);
                    mres_cycle(st, n, gm, ls, d_mask, mr_mu, (double *const *)p_x64, mr_sc, false);
                    mres_init(st, n, gm, ls, d_mask, mr_ext, mr_sc, ls.active);
                };
                cycle_start(act);
                if (per_rhs) {
                    // the guess from range(U_j) alone: its residual is the first cycle's xi
                    std::vector<double> sc0((size_t)m * MR_NSC);
                    c->d2h(sc0.data(), mr_sc, sc0.size());
                    c->sync();
                    for (int l = 0; l < m; ++l)
                        if (act[l]) out[l].relres0 = relres0[l] = sc0[(size_t)l * MR_NSC + MR_XI] / std::fabs(lw[l]);
                }
                while (true) {
                    for (int i = 0; i < chunk; ++i)
                        mres_iteration(st, g, (const double *)D, (const double *const *)p_diag,
                                       (const double *const *)p_p, (double *const *)p_q, gm, ls, ls.active, mr_step,
                                       mr_alpha, mr_hd, mr_mu, mr_ext, mr_sc);
                    c->d2h(flag_h.data(), ls.flag, m);
                    c->d2h(active_h.data(), ls.active, m);
                    c->d2h(iters_h.data(), ls.iters, m);
                    c->sync();
                    std::vector<int> F;
                    for (int l = 0; l < m; ++l)
                        if (act[l] && !done[l] && (flag_h[l] != 0 || !active_h[l])) F.push_back(l);
                    if (!F.empty()) {
                        // end of the cycle: x += y - W H^-1 (A~W)^T A~ y, then the float64 residual
                        std::vector<int> fmask(m, 0);
                        for (int l : F) fmask[l] = 1;
                        c->h2d(d_mask, fmask.data(), m);
                        apply_op<double>(st, g, c->D64, (const double *const *)p_diag64, (const double *const *)p_xc,
                                         (double *const *)p_q, m, d_mask, nullptr, nullptr);
                        mres_dots(st, n, gq, ls, d_mask, (const double *)gm.q, mr_hd);
                        mres_mu(st, ls, d_mask, mr_hd, mr_mu, mr_sc);
                        mres_cycle(st, n, gm, ls, d_mask, mr_mu, (double *const *)p_x64, mr_sc, true);
                        residual(rr_h, d_mask, (int)F.size());
                        std::vector<int> Rl, rmask(m, 0);
                        for (int l : F) {
                            relres[l] = std::sqrt(rr_h[l]) / std::fabs(lw[l]);
                            if (relres[l] <= ltol[l]) done[l] = 1;
                            else if (iters_h[l] >= c->opt.maxit || restarts[l] > 200) {
                                done[l] = 1;
                                status[l] = RCG_ERR_NOT_CONVERGED;
                            } else {
                                Rl.push_back(l);
                                rmask[l] = 1;
                                ++restarts[l];
                            }
                        }
                        if (!Rl.empty()) {
                            RCG_CUDA_TRY(cudaMemsetAsync(ls.flag, 0, sizeof(int) * m, st));
                            cycle_start(rmask);
                        }
                    }
                    bool any = false;
                    for (int l = 0; l < m; ++l)
                        if (act[l] && !done[l]) any = true;
                    if (!any) break;
                }
                if (per_rhs) {
                    std::vector<int> sel(m, 0);
                    for (int l = 0; l < m; ++l) sel[l] = act[l] && status[l] == RCG_OK;
                    per_rhs_store(sel, lanes, gm, c->opt.tau_rank, prh_kept);
                }
            } else {
            restart(act);
            // RCG_LEARN_START: the learned columns are gone after the first
            // start, so the iterations take the templates of the other columns
            if (c->opt.learned_mode == RCG_LEARN_START) gm.kp_sel = std::max(kp_max, 1);
            if (vec) build_list();
            while (true) {
                if (graph) {
                    if (!cgg.ready())
                        cgg.capture([&](cudaStream_t cs) {
                            for (int i = 1; i <= chunk; ++i)
                                cg_iteration<T>(cs, g, D, (const T *const *)p_diag, (const T *const *)p_p, p_q, gm, ls,
                                                t + i, nullptr);
                        });
                    cgg.launch();
                    t += chunk;
                } else {
                    for (int i = 0; i < chunk; ++i) {
                        ++t;
                        if (vec)
                            cg_iteration4(st, g, (const float *)D, (const float *const *)p_diag,
                                          (const float *const *)p_p, (float *const *)p_q, gm, ls, ll, t, mu_f, beta_f,
                                          &c->ktimer);
                        else
                            cg_iteration<T>(st, g, D, (const T *const *)p_diag, (const T *const *)p_p, p_q, gm, ls, t,
                                            &c->ktimer);
                    }
                }
                c->d2h(flag_h.data(), ls.flag, m);
                c->d2h(active_h.data(), ls.active, m);
                c->d2h(iters_h.data(), ls.iters, m);
                c->sync();
                c->ktimer.harvest();
                if (vec && stencil_take_error(st))
                    throw Error{RCG_ERR_TIMEOUT, "stencil: a TMA copy's wait ran out"};
                std::vector<int> F;
                bool force = false;
                for (int l = 0; l < m; ++l) {
                    if (!act[l] || done[l]) continue;
                    if (flag_h[l] != 0 || !active_h[l]) F.push_back(l);
                    else if (iters_h[l] >= c->opt.maxit) { F.push_back(l); force = true; }
                }
                if (force) {   // stop lanes over maxit
                    std::vector<int> zero_act(active_h);
                    for (int l : F) zero_act[l] = 0;
                    c->h2d(ls.active, zero_act.data(), m);
                }
                if (!F.empty()) {
                    std::vector<int> fmask(m, 0);
                    for (int l : F) fmask[l] = 1;
                    c->h2d(d_list, F.data(), F.size());
                    c->h2d(d_mask, fmask.data(), m);
                    dim3 gr((unsigned)std::min<long long>((n + 255) / 256, 512), (unsigned)F.size());
                    k_add_lanes<T><<<gr, 256, 0, st>>>(n, x64, ld, xc, ld, d_list);
                    ++c->launches;
                    RCG_CHECK_LAUNCH();
                    residual(rr_h, d_mask, (int)F.size());
                    std::vector<int> Rl;
                    for (int l : F) {
                        relres[l] = std::sqrt(rr_h[l]) / std::fabs(lw[l]);
                        if (relres[l] <= ltol[l]) { done[l] = 1; }
                        else if (iters_h[l] >= c->opt.maxit) { done[l] = 1; status[l] = RCG_ERR_NOT_CONVERGED; }
                        else if (restarts[l] > 200) { done[l] = 1; status[l] = RCG_ERR_NOT_CONVERGED; }
                        else { Rl.push_back(l); ++restarts[l]; set_thresh(l, std::sqrt(rr_h[l])); }
                    }
                    if (!Rl.empty()) {
                        std::vector<int> rmask(m, 0);
                        for (int l : Rl) rmask[l] = 1;
                        c->h2d(ls.thresh, thr.data(), m);
                        c->h2d(d_mask, rmask.data(), m);
                        restart(rmask);
                    }
                }
                bool any = false;
                for (int l = 0; l < m; ++l)
                    if (act[l] && !done[l]) any = true;
                if (!any) break;
                if (vec) build_list();
            }
            }
            c->d2h(iters_h.data(), ls.iters, m);
            c->sync();
            if (net && net->record && !alanes.empty()) {
                // training pairs: features of r0 and coarse(x - x0) / max, x the delivered solution
                const int na = (int)alanes.size();
                net->pool64(st, d_lx, net->x0c, na, 1.f, true);
                net->normalise(st, net->x0c, na);
                net->add_pairs(st, net->feat, net->x0c, na);
            }
        }
        RCG_CUDA_TRY(cudaEventRecord(e2, st));

        // ---- ordered append of the new solutions
        std::vector<int> cand;
        for (int l = 0; l < m; ++l)
            if (seed_mode || (act[l] && status[l] == RCG_OK)) cand.push_back(l);
        std::vector<int> kept;
        std::vector<double> ratio;
        const int r_before = r;
        if (per_rhs) {
            kept.assign(cand.size(), 0);
            ratio.assign(cand.size(), 0.0);
            for (size_t ci = 0; ci < cand.size(); ++ci) kept[ci] = prh_kept.empty() ? 0 : prh_kept[cand[ci]];
        } else {
            append(cand, tau, (seq && !seed_mode) ? lanes[0].s : -1, kept, ratio);
        }
        int qi = 0;
        for (size_t ci = 0; ci < cand.size(); ++ci) {
            const int l = cand[ci];
            out[l].ratio = ratio[ci];
            out[l].appended = kept[ci];
            if (kept[ci] && !seed_mode && !per_rhs) {
                auto &pl = priv[lanes[l].j];
                pl.push_back(r_before + qi);
                while (k_u + (int)pl.size() > std::min(c->opt.k_cap, k_u + KP_MAX) && !pl.empty()) pl.erase(pl.begin());
            }
            if (kept[ci]) ++qi;
        }
        RCG_CUDA_TRY(cudaEventRecord(e3, st));
        c->sync();
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1); c->phase["check"] += ms;
        cudaEventElapsedTime(&ms, e1, e2); c->phase["cg"] += ms;
        cudaEventElapsedTime(&ms, e2, e3); c->phase["append"] += ms;
        cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2); cudaEventDestroy(e3);
        for (int l = 0; l < m; ++l) {
            out[l].iters = act[l] ? iters_h[l] : 0;
            out[l].restarts = restarts[l];
            out[l].relres = relres[l];
            out[l].status = status[l];
        }
        if (c->opt.keep_solutions) {
            // with D tracking mu the lanes solved with the reference weights: scale each
            // solution by the ratio of its sample's weight to the reference one
            double *ws = nullptr, *xs = nullptr;
            if (c->track()) {
                ws = c->alloc<double>((size_t)c->nrhs);
                xs = c->alloc<double>(ld);
            }
            int ws_sample = -1;
            for (int l = 0; l < m; ++l) {
                auto &sol = c->solutions[lanes[l].s];
                if (sol.empty()) sol.assign((size_t)n * c->nrhs, 0.0);
                const double *src = x64 + (long long)l * ld;
                if (c->track()) {
                    if (ws_sample != lanes[l].s) {
                        rhs_weights(st, c->Ds64_of(lanes[l].s), c->d_rhs_node, c->d_rhs_wt, c->nsrc, c->nrhs,
                                    c->grid.robin_A, c->h, ws);
                        ws_sample = lanes[l].s;
                    }
                    ratio_scale(st, n, src, ld, ws + lanes[l].j, c->d_rhs_w + lanes[l].j, xs, ld, 1);
                    src = xs;
                }
                c->d2h(sol.data() + (size_t)lanes[l].j * n, src, n);
            }
            c->sync();
            c->release(ws);
            c->release(xs);
        }
    }

    // -------------------------------------------------------------- seed
    // CholQR of the b columns of X (twice), using Y as scratch.
    void cholqr(T *X, T *Y, int b) {
        for (int pass = 0; pass < 2; ++pass) {
            prod_tn(X, b, X, b, M, b, true);
            RCG_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), st));
            chol_inplace(st, M, b, b, d_info);
            check_info("eigen seed CholQR");
            lower_to_upper(st, M, b, b, RK);
            tri_upper_inverse(st, RK, b, b, Ri);
            prod_nn(X, b, Ri, b, b, Y, 1.0, 0.0);
            RCG_CUDA_TRY(cudaMemcpyAsync(X, Y, sizeof(T) * (size_t)b * ld, cudaMemcpyDeviceToDevice, st));
        }
    }

    // Rayleigh-Ritz on range(X): X <- Ritz vectors (ascending), AX = A~ X, theta.
    void rayleigh_ritz(int s0, T *X, T *AX, T *Y, int b, std::vector<double> &theta) {
        std::vector<const T *> src(b);
        std::vector<T *> dst(b);
        for (int i = 0; i < b; ++i) { src[i] = X + (long long)i * ld; dst[i] = AX + (long long)i * ld; }
        apply_cols(src, dst, std::vector<int>(b, s0));
        prod_tn(X, b, AX, b, M, b);
        jacobi_eig(st, M, b, b, Rhat, xn2);          // Rhat: eigenvectors, xn2: eigenvalues
        prod_nn(X, b, Rhat, b, b, Y, 1.0, 0.0);
        RCG_CUDA_TRY(cudaMemcpyAsync(X, Y, sizeof(T) * (size_t)b * ld, cudaMemcpyDeviceToDevice, st));
        prod_nn(AX, b, Rhat, b, b, Y, 1.0, 0.0);
        RCG_CUDA_TRY(cudaMemcpyAsync(AX, Y, sizeof(T) * (size_t)b * ld, cudaMemcpyDeviceToDevice, st));
        theta.resize(b);
        c->d2h(theta.data(), xn2, b);
        c->sync();
    }

    // k_u smallest eigenvectors of A~_{s0} by Chebyshev-filtered subspace
    // iteration (Zhou & Saad 2007) with block size k_u + 6: each pass filters
    // the block with a Chebyshev polynomial damping [a, lambda_max] (a = the
    // largest Ritz value of the block, lambda_max a Gershgorin bound), then
    // orthonormalises and does a Rayleigh-Ritz step.  Result: x64 lanes 0..k_u-1.
    void seed_eig(int s0) {
        const int b = std::min(k_u + 6, 32);
        ensure_lanes(std::max(c->nrhs, b));
        ensure_append(b);
        T *X = xc, *AX = rv, *Y1 = pv, *Y2 = qv;
        unsigned long long *gb = (unsigned long long *)d_rr;
        gershgorin(st, g, sample_D(g, c->diag64_of(s0), c->D64), c->diag64_of(s0), gb);
        unsigned long long bits = 0;
        c->d2h(&bits, gb, 1);
        c->sync();
        double lmax;
        std::memcpy(&lmax, &bits, sizeof(double));
        rand_fill<T>(st, X, n, ld, b, 0x5EED5EEDULL);
        cholqr(X, Y1, b);
        std::vector<double> theta, res(b);
        rayleigh_ritz(s0, X, AX, Y1, b, theta);
        const int degree = c->opt.seed_degree > 0 ? c->opt.seed_degree : 24;
        const double tol = mixed ? 3e-6 : 1e-10;
        double *res_d = d_rr;
        for (int pass = 0; pass < 400; ++pass) {
            const double a = theta[b - 1];
            const double e = 0.5 * (lmax - a), cc = 0.5 * (lmax + a);
            // Y1 = (A X - c X) / e ; Y_{k+1} = 2 (A Y_k - c Y_k)/e - Y_{k-1}
            std::vector<const T *> src(b);
            std::vector<T *> dst(b);
            T *buf[3] = {X, Y1, Y2};      // Y_k lives in buf[k mod 3]
            for (int k = 0; k < degree; ++k) {
                T *Yk = buf[k % 3], *Ykm1 = buf[(k + 2) % 3], *Ynew = buf[(k + 1) % 3];
                for (int i = 0; i < b; ++i) { src[i] = Yk + (long long)i * ld; dst[i] = AX + (long long)i * ld; }
                apply_cols(src, dst, std::vector<int>(b, s0));
                if (k == 0) cheb_step<T>(st, Ynew, AX, Yk, nullptr, n, ld, b, 1.0 / e, -cc / e, 0.0);
                else cheb_step<T>(st, Ynew, AX, Yk, Ykm1, n, ld, b, 2.0 / e, -2.0 * cc / e, -1.0);
            }
            if (degree % 3 != 0)
                RCG_CUDA_TRY(cudaMemcpyAsync(X, buf[degree % 3], sizeof(T) * (size_t)b * ld, cudaMemcpyDeviceToDevice, st));
            cholqr(X, Y1, b);
            rayleigh_ritz(s0, X, AX, Y1, b, theta);
            ritz_res<T>(st, AX, X, xn2, n, ld, b, res_d);
            c->d2h(res.data(), res_d, b);
            c->sync();
            double worst = 0;
            for (int i = 0; i < k_u; ++i) worst = std::max(worst, std::sqrt(res[i]));
            if (worst <= tol * lmax) break;
        }
        for (int i = 0; i < k_u; ++i)
            convert_cols<T, double>(st, n, X + (long long)i * ld, ld, x64 + (long long)i * ld, ld, 1);
        c->sync();
    }

    void seed(int s0, const double *U0, rcg_stat *stats) override {
        au0_valid = false;
        s_star = s0;
        r = 0;
        gs_sample = -1;
        k_u = c->opt.k_u;
        const int nrhs = c->nrhs;
        ensure_lanes(std::max(nrhs, k_u));
        // U_0 -> V through the append (orthonormalises in order)
        if (k_u > 0) {
            cudaEvent_t e0, e1;
            RCG_CUDA_TRY(cudaEventCreate(&e0)); RCG_CUDA_TRY(cudaEventCreate(&e1));
            RCG_CUDA_TRY(cudaEventRecord(e0, st));
            if (U0) {
                for (int q = 0; q < k_u; ++q) c->h2d(x64 + (long long)q * ld, U0 + (size_t)q * n, n);
            } else {
                seed_eig(s0);
            }
            RCG_CUDA_TRY(cudaEventRecord(e1, st));
            c->sync();
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaEventDestroy(e0); cudaEventDestroy(e1);
            c->phase.clear();
            c->phase["seed_eig"] = ms;
            std::vector<int> cand(k_u);
            for (int q = 0; q < k_u; ++q) cand[q] = q;
            std::vector<int> kept;
            std::vector<double> ratio;
            append(cand, 1e-12, -1, kept, ratio);
            k_u = r;
        }
        // X_0 = A~_0^-1 [B~, C~] by deflated CG with U_0, appended in RHS order
        std::vector<Lane> lanes(nrhs);
        for (int j = 0; j < nrhs; ++j) lanes[j] = Lane{s0, j};
        if (!X0) { X0 = c->alloc<T>((size_t)nrhs * ld); sX0 = c->alloc<double>((size_t)rmax * nrhs); }
        priv.assign(nrhs, {});
        std::vector<rcg_stat> out;
        const double eig_ms = c->phase.count("seed_eig") ? c->phase["seed_eig"] : 0.0;
        c->phase.clear();
        c->phase["seed_eig"] = eig_ms;
        wave(lanes, true, false, out);
        c->phase["seed_x0"] = c->phase["check"] + c->phase["cg"] + c->phase["append"];
        std::vector<int> all(nrhs);
        for (int j = 0; j < nrhs; ++j) all[j] = j;
        c->h2d(d_list, all.data(), nrhs);
        convert_lanes<double, T>(st, n, (const double *const *)p_x64, d_list, nrhs, X0, ld);
        RCG_CUDA_TRY(cudaMemsetAsync(sX0, 0, sizeof(double) * rmax * nrhs, st));
        prod_tn(V, r, X0, nrhs, sX0, rmax);
        c->sync();
        priv.assign(nrhs, std::vector<int>{-1});
        priv_seed = priv;
        r_seed = r;
        seeded = true;
        if (stats) for (int j = 0; j < nrhs; ++j) stats[j] = out[j];
    }

    SeedView seed_view() const override {
        SeedView sv;
        sv.seeded = seeded;
        sv.esize = (int)sizeof(T);
        sv.r_seed = r_seed;
        sv.k_u = k_u;
        sv.s_star = s_star;
        sv.rmax = rmax;
        sv.V = V;
        sv.X0 = X0;
        sv.Cstar = Cstar;
        sv.priv_seed = priv_seed;
        return sv;
    }

    // The seed state of another engine: V's first r_seed columns, the leading
    // block of C_* (exact: float32 values are exact in float64), X_0 and the
    // recycle lists; V^T X_0 recomputed in this engine's arithmetic.
    void seed_import(const SeedView &sv) override {
        if (!sv.seeded) throw Error{RCG_ERR_INVALID, "rcg_seed_copy: the source context is not seeded"};
        if (sv.esize != (int)sizeof(T) && !(sv.esize == 4 && sizeof(T) == 8))
            throw Error{RCG_ERR_INVALID, "rcg_seed_copy: a float64 seed cannot go into a float32 context"};
        if (sv.r_seed > rmax) throw Error{RCG_ERR_RANK_CAP, "rcg_seed_copy: the seed basis exceeds r_max"};
        const int nrhs = c->nrhs;
        r = 0;
        ensure_vcap(sv.r_seed);
        if (!X0) { X0 = c->alloc<T>((size_t)nrhs * ld); sX0 = c->alloc<double>((size_t)rmax * nrhs); }
        if (sv.esize == (int)sizeof(T)) {
            RCG_CUDA_TRY(cudaMemcpyAsync(V, sv.V, sizeof(T) * (size_t)sv.r_seed * ld, cudaMemcpyDeviceToDevice, st));
            RCG_CUDA_TRY(cudaMemcpyAsync(X0, sv.X0, sizeof(T) * (size_t)nrhs * ld, cudaMemcpyDeviceToDevice, st));
        } else {
            convert_cols<float, T>(st, n, (const float *)sv.V, ld, V, ld, sv.r_seed);
            convert_cols<float, T>(st, n, (const float *)sv.X0, ld, X0, ld, nrhs);
        }
        RCG_CUDA_TRY(cudaMemcpy2DAsync(Cstar, sizeof(double) * rmax, sv.Cstar, sizeof(double) * sv.rmax,
                                       sizeof(double) * sv.r_seed, sv.r_seed, cudaMemcpyDeviceToDevice, st));
        r = sv.r_seed;
        RCG_CUDA_TRY(cudaMemsetAsync(sX0, 0, sizeof(double) * rmax * nrhs, st));
        prod_tn(V, r, X0, nrhs, sX0, rmax);
        c->sync();
        r_seed = r;
        k_u = sv.k_u;
        s_star = sv.s_star;
        priv = priv_seed = sv.priv_seed;
        gs_sample = -1;
        au0_valid = false;
        for (auto &d : dw_star) d = -1;
        seeded = true;
    }

    void reset() override {
        if (!seeded) throw Error{RCG_ERR_INVALID, "rcg_reset_to_seed before rcg_seed"};
        r = r_seed;
        priv = priv_seed;
        gs_sample = -1;
    }

    // ---------------------------------------------------------- Algorithm 1
    // Steps 2-3 of Algorithm 1 on the delivered solutions kept so far
    // (samples in ascending order): S = [X_s1, X_s2, ...] (n x m), the Gram
    // S^T S in float64, its eigen-decomposition by the parallel Jacobi method,
    // sigma_i = sqrt(lambda_i), and V <- S W_r diag(sigma)^-1 for the r =
    // min(r_cap, #{sigma_i > tau sigma_1}) leading pairs, passed through the
    // ordered append (re-orthonormalised, C_* rebuilt).  The shared deflation
    // space becomes the leading min(k_u, r) columns and the private recycle
    // lists restart empty (X_0 need not lie in the truncated range(V), and a
    // private column's deflation matrix is formed through V^T x); the seed
    // state becomes the compressed basis.
    // Returns the number of snapshot columns m; sigma gets all m values.
    int compress(int r_cap, double tau, std::vector<double> &sigma) override {
        if (!seeded) throw Error{RCG_ERR_INVALID, "rcg_basis_compress before rcg_seed"};
        if (!c->opt.keep_solutions) throw Error{RCG_ERR_INVALID, "rcg_basis_compress needs options.keep_solutions"};
        std::vector<int> samp;
        for (int s = 0; s < c->opt.max_samples; ++s)
            if (!c->solutions[s].empty()) samp.push_back(s);
        if (samp.empty()) throw Error{RCG_ERR_INVALID, "rcg_basis_compress: no delivered solutions are kept"};
        const int nrhs = c->nrhs;
        const int m = (int)samp.size() * nrhs, m2 = m + (m & 1);
        // the Gram eigensolver costs O(m^3) float64 operations per sweep (~4 s at m = 4096)
        if (m > RCG_COMPRESS_MAX_COLS)
            throw Error{RCG_ERR_INVALID, "rcg_basis_compress: more than RCG_COMPRESS_MAX_COLS snapshot columns kept"};
        if (r_cap <= 0 || r_cap > rmax) r_cap = rmax;
        cudaEvent_t e0, e1;
        RCG_CUDA_TRY(cudaEventCreate(&e0)); RCG_CUDA_TRY(cudaEventCreate(&e1));
        RCG_CUDA_TRY(cudaEventRecord(e0, st));
        double *S = c->alloc<double>((size_t)m * ld);
        double *M = c->alloc<double>((size_t)m2 * m2), *E = c->alloc<double>((size_t)m2 * m2);
        double *cs = c->alloc<double>((size_t)m2), *red = c->alloc<double>(2);
        double *Wr = nullptr;
        try {
            for (size_t b = 0; b < samp.size(); ++b)
                for (int j = 0; j < nrhs; ++j)
                    c->h2d(S + ((long long)b * nrhs + j) * ld, c->solutions[samp[b]].data() + (size_t)j * n, (size_t)n);
            RCG_CUDA_TRY(cudaMemsetAsync(M, 0, sizeof(double) * (size_t)m2 * m2, st));   // odd m: zero last row / column
            gemm_tn<double, double>(st, n, S, ld, m, S, ld, m, M, m2, false);
            jacobi_parallel(st, M, m2, m2, E, m2, cs, red, 1e-14, 40);
            std::vector<double> lam((size_t)m2), Eh((size_t)m2 * m2);
            RCG_CUDA_TRY(cudaMemcpy2DAsync(lam.data(), sizeof(double), M, sizeof(double) * (m2 + 1), sizeof(double), m2,
                                           cudaMemcpyDeviceToHost, st));
            c->d2h(Eh.data(), E, (size_t)m2 * m2);
            c->sync();
            std::vector<int> idx((size_t)m2);
            for (int i = 0; i < m2; ++i) idx[i] = i;
            std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return lam[a] > lam[b]; });
            sigma.assign((size_t)m, 0.0);
            for (int i = 0; i < m; ++i) sigma[i] = std::sqrt(std::max(lam[idx[i]], 0.0));
            int rn = 0;
            if (sigma[0] > 0.0)
                while (rn < m && sigma[rn] > tau * sigma[0]) ++rn;
            rn = std::min(rn, r_cap);
            if (rn == 0) throw Error{RCG_ERR_INVALID, "rcg_basis_compress: no singular value above tau sigma_1"};
            // W_r diag(sigma)^-1 (m x rn), then the new columns into the lane buffers
            std::vector<double> wr((size_t)m * rn);
            for (int q = 0; q < rn; ++q)
                for (int i = 0; i < m; ++i) wr[(size_t)q * m + i] = Eh[(size_t)idx[q] * m2 + i] / sigma[q];
            Wr = c->alloc<double>((size_t)m * rn);
            c->h2d(Wr, wr.data(), wr.size());
            ensure_lanes(rn);
            gemm_nn<double, double>(st, n, S, ld, m, Wr, m, rn, x64, ld, 1.0, 0.0);
            // rebuild V (and C_*) from these columns
            r = 0;
            gs_sample = -1;
            au0_valid = false;
            std::vector<int> cand((size_t)rn), kept;
            std::vector<double> ratio;
            for (int q = 0; q < rn; ++q) cand[q] = q;
            append(cand, 1e-12, -1, kept, ratio);
            k_u = std::min(k_u, r);
            RCG_CUDA_TRY(cudaMemsetAsync(sX0, 0, sizeof(double) * rmax * nrhs, st));
            prod_tn(V, r, X0, nrhs, sX0, rmax);
            priv.assign(nrhs, std::vector<int>{});
            priv_seed = priv;
            r_seed = r;
        } catch (...) {
            for (void *q : std::vector<void *>{S, M, E, cs, red, Wr}) c->release(q);
            cudaEventDestroy(e0); cudaEventDestroy(e1);
            throw;
        }
        RCG_CUDA_TRY(cudaEventRecord(e1, st));
        c->sync();
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        c->phase["compress"] = ms;
        cudaEventDestroy(e0); cudaEventDestroy(e1);
        for (void *q : std::vector<void *>{S, M, E, cs, red, Wr}) c->release(q);
        return m;
    }

    int solve_all(int s_first, int s_count, rcg_stat *stats) override {
        if (!seeded) throw Error{RCG_ERR_INVALID, "rcg_solve_all before rcg_seed"};
        const int nrhs = c->nrhs;
        int rc = RCG_OK;
        c->phase.erase("check"); c->phase.erase("cg"); c->phase.erase("append");
        c->phase["check"] = c->phase["cg"] = c->phase["append"] = 0.0;
        auto record = [&](const std::vector<rcg_stat> &out) {
            for (const auto &o : out) {
                if (o.status == RCG_ERR_NOT_CONVERGED && rc == RCG_OK) rc = RCG_ERR_NOT_CONVERGED;
                if (o.status == RCG_ERR_BREAKDOWN && rc == RCG_OK) rc = RCG_ERR_BREAKDOWN;
                if (stats) stats[(size_t)(o.sample - s_first) * nrhs + o.rhs] = o;
            }
        };
        std::vector<rcg_stat> out;
        if (c->opt.order == RCG_SEQUENTIAL) {
            for (int s = s_first; s < s_first + s_count; ++s)
                for (int j = 0; j < nrhs; ++j) {
                    wave({Lane{s, j}}, false, true, out);
                    record(out);
                }
        } else {
            // waves: `wave_samples` samples x `wave_rhs` consecutive RHS; the
            // RHS blocks of a sample group run one after another, each seeing
            // the columns the earlier blocks appended (the paper's inner-outer
            // effect, kept in blocks of batched lanes)
            const int ws = c->opt.wave_samples > 0 ? c->opt.wave_samples : s_count;
            const int wr = c->opt.wave_rhs > 0 ? std::min(c->opt.wave_rhs, nrhs) : nrhs;
            for (int s0 = s_first; s0 < s_first + s_count; s0 += ws)
                for (int j0 = 0; j0 < nrhs; j0 += wr) {
                    std::vector<Lane> lanes;
                    for (int s = s0; s < std::min(s0 + ws, s_first + s_count); ++s)
                        for (int j = j0; j < std::min(j0 + wr, nrhs); ++j) lanes.push_back(Lane{s, j});
                    wave(lanes, false, false, out);
                    record(out);
                }
        }
        return rc;
    }

    // ---------------------------------------------------------- state I/O
    // The recycling state: V (r columns), C_* = V^T A~_* V, X_0 and V^T X_0,
    // the private recycle lists and the state right after the seed.
    void save(std::FILE *f) override {
        if (!seeded) throw Error{RCG_ERR_INVALID, "rcg_save before rcg_seed"};
        const long long hdr[6] = {(long long)sizeof(T), r, r_seed, s_star, k_u, c->nrhs};
        wr(f, hdr, sizeof(hdr));
        std::vector<T> hv((size_t)r * n);
        for (int q = 0; q < r; ++q) c->d2h(hv.data() + (size_t)q * n, V + (long long)q * ld, (size_t)n);
        std::vector<double> hc((size_t)r * r);
        RCG_CUDA_TRY(cudaMemcpy2DAsync(hc.data(), sizeof(double) * r, Cstar, sizeof(double) * rmax, sizeof(double) * r,
                                       r, cudaMemcpyDeviceToHost, st));
        std::vector<T> hx((size_t)c->nrhs * n);
        for (int j = 0; j < c->nrhs; ++j) c->d2h(hx.data() + (size_t)j * n, X0 + (long long)j * ld, (size_t)n);
        std::vector<double> hs((size_t)r * c->nrhs);
        RCG_CUDA_TRY(cudaMemcpy2DAsync(hs.data(), sizeof(double) * r, sX0, sizeof(double) * rmax, sizeof(double) * r,
                                       c->nrhs, cudaMemcpyDeviceToHost, st));
        c->sync();
        wr_vec(f, hv);
        wr_vec(f, hc);
        wr_vec(f, hx);
        wr_vec(f, hs);
        for (auto *pl : {&priv, &priv_seed})
            for (int j = 0; j < c->nrhs; ++j) wr_vec(f, (*pl)[j]);
        // mu_* of the seed sample, which C_* belongs to
        std::vector<double> mu((size_t)n);
        c->d2h(mu.data(), c->mu64 + (long long)s_star * ld, (size_t)n);
        c->sync();
        wr_vec(f, mu);
    }

    void load(std::FILE *f) override {
        long long hdr[6];
        rd(f, hdr, sizeof(hdr));
        if (hdr[0] != (long long)sizeof(T) || hdr[5] != c->nrhs || hdr[1] < 0 || hdr[1] > rmax || hdr[2] < 0 ||
            hdr[2] > hdr[1] || hdr[3] < 0 || hdr[3] >= c->opt.max_samples)
            throw Error{RCG_ERR_INVALID, "rcg_load: precision, RHS count or basis size does not match the context"};
        const int rr = (int)hdr[1], nrhs = c->nrhs;
        auto hv = rd_vec<T>(f, (long long)rr * n);
        auto hc = rd_vec<double>(f, (long long)rr * rr);
        auto hx = rd_vec<T>(f, (long long)nrhs * n);
        auto hs = rd_vec<double>(f, (long long)rr * nrhs);
        if ((long long)hv.size() != (long long)rr * n || (long long)hc.size() != (long long)rr * rr ||
            (long long)hx.size() != (long long)nrhs * n || (long long)hs.size() != (long long)rr * nrhs)
            throw Error{RCG_ERR_INVALID, "rcg_load: array sizes do not match the context"};
        std::vector<std::vector<int>> p1(nrhs), p2(nrhs);
        for (auto *pl : {&p1, &p2})
            for (int j = 0; j < nrhs; ++j) {
                (*pl)[j] = rd_vec<int>(f, KP_MAX + 1);
                for (int e : (*pl)[j])
                    if (e < -1 || e >= rr) throw Error{RCG_ERR_INVALID, "rcg_load: bad recycle list"};
            }
        auto mu = rd_vec<double>(f, n);
        if ((long long)mu.size() != n) throw Error{RCG_ERR_INVALID, "rcg_load: mu_* size"};
        ensure_lanes(std::max(nrhs, 1));
        if (!X0) { X0 = c->alloc<T>((size_t)nrhs * ld); sX0 = c->alloc<double>((size_t)rmax * nrhs); }
        // the seed sample slot gets mu_* back (its diagonal too)
        const int ss = (int)hdr[3];
        c->h2d(c->mu64 + (long long)ss * ld, mu.data(), (size_t)n);
        if (c->track())
            track_coefficients(st, g, c->mu64 + (long long)ss * ld, c->opt.mu_s_prime, c->h, c->grid.robin_A,
                               c->Ds64_of(ss), c->Ds32 + (long long)ss * ld, c->Ws64_of(ss), c->diag64_of(ss),
                               c->diag32_of(ss));
        else
            diag_sample(st, n, c->dstar, c->mu64 + (long long)ss * ld, c->h * c->h, c->diag64_of(ss),
                        c->diag32_of(ss));
        c->sample_set[ss] = 1;
        r = 0;
        ensure_vcap(rr);
        for (int q = 0; q < rr; ++q) c->h2d(V + (long long)q * ld, hv.data() + (size_t)q * n, (size_t)n);
        RCG_CUDA_TRY(cudaMemcpy2DAsync(Cstar, sizeof(double) * rmax, hc.data(), sizeof(double) * rr, sizeof(double) * rr,
                                       rr, cudaMemcpyHostToDevice, st));
        for (int j = 0; j < nrhs; ++j) c->h2d(X0 + (long long)j * ld, hx.data() + (size_t)j * n, (size_t)n);
        RCG_CUDA_TRY(cudaMemsetAsync(sX0, 0, sizeof(double) * rmax * nrhs, st));
        RCG_CUDA_TRY(cudaMemcpy2DAsync(sX0, sizeof(double) * rmax, hs.data(), sizeof(double) * rr, sizeof(double) * rr,
                                       nrhs, cudaMemcpyHostToDevice, st));
        c->sync();
        r = rr;
        r_seed = (int)hdr[2];
        s_star = (int)hdr[3];
        k_u = (int)hdr[4];
        priv = p1;
        priv_seed = p2;
        gs_sample = -1;
        au0_valid = false;
        for (auto &d : dw_star) d = -1;
        seeded = true;
    }

    int rank() const override { return r; }

    // caches derived from mu_s: Delta weights, A~_s U_0, the sequential G_s
    void sample_changed(int s) override {
        if (s >= 0 && s < (int)dw_star.size()) dw_star[s] = -1;
        if (std::find(au0_samples.begin(), au0_samples.end(), s) != au0_samples.end()) au0_valid = false;
        if (gs_sample == s) gs_sample = -1;
        if (s == s_star) seeded = false;     // C_* and the seed belong to the old mu_*: seed again
    }

    void basis_get(double *Vh) override {
        if (r == 0) return;
        double *tmp = c->alloc<double>((size_t)r * ld);
        convert_cols<T, double>(st, n, V, ld, tmp, ld, r);
        RCG_CUDA_TRY(cudaMemcpy2DAsync(Vh, sizeof(double) * n, tmp, sizeof(double) * ld, sizeof(double) * n, r,
                                       cudaMemcpyDeviceToHost, st));
        c->sync();
        c->release(tmp);
    }

    // ----------------------------------------------------------- reduced model
    void rom_eval(const double *mu, int nparam, const double *dmu, double *Psi, double *J) override {
        if (r == 0) throw Error{RCG_ERR_INVALID, "rcg_rom_eval with an empty basis"};
        const int ns = c->nsrc, nd = c->ndet;
        cudaEvent_t e0, e1;
        RCG_CUDA_TRY(cudaEventCreate(&e0)); RCG_CUDA_TRY(cudaEventCreate(&e1));
        RCG_CUDA_TRY(cudaEventRecord(e0, st));
        if (!Ar) {
            Ar = c->alloc<double>((size_t)rmax * rmax);
            Br = c->alloc<double>((size_t)rmax * ns);
            Crm = c->alloc<double>((size_t)rmax * nd);
            Xr = c->alloc<double>((size_t)rmax * ns);
            Zr = c->alloc<double>((size_t)rmax * nd);
            wtmp = c->alloc<double>(ld);
        }
        // A~_r = C_* + V^T (A~(p) - A~_*) V
        RCG_CUDA_TRY(cudaMemcpy2DAsync(Ar, sizeof(double) * r, Cstar, sizeof(double) * rmax, sizeof(double) * r, r,
                                       cudaMemcpyDeviceToDevice, st));
        const double *wsrc = c->d_rhs_w;                   // effective source / detector weights at p
        if (c->track()) {
            ensure_track();
            if (!tp_D) {
                tp_D = c->alloc<double>(ld);
                tp_W = c->alloc<double>((size_t)3 * ld);
                tp_diag = c->alloc<double>(ld);
                tp_w = c->alloc<double>(c->nrhs);
                tp_G = c->alloc<double>((size_t)rmax * c->nrhs);
                tp_P = c->alloc<double>((size_t)2 * ns * nd);
            }
            track_coefficients(st, g, mu, c->opt.mu_s_prime, c->h, c->grid.robin_A, tp_D, nullptr, tp_W, tp_diag,
                               nullptr);
            scaled_diff(st, n, tp_diag, c->diag64_of(s_star), 1.0, tk_dg);
            scaled_diff(st, 3 * ld, tp_W, c->Ws64_of(s_star), 1.0, tk_dw);
            delta_gram(V, r, Ar, r);
            rhs_weights(st, tp_D, c->d_rhs_node, c->d_rhs_wt, ns, c->nrhs, c->grid.robin_A, c->h, tp_w);
            wsrc = tp_w;
        } else {
            scaled_diff(st, n, mu, c->mu64 + (long long)s_star * ld, c->h * c->h, wtmp);
            if (mixed) {
                if (!rom_bl) { rom_bl = c->alloc<int>((size_t)(n + 31) / 32); rom_bc = c->alloc<int>(1); }
                tc_block_list(st, n, wtmp, rom_bl, rom_bc);
            }
            gram_w_acc(V, r, Ar, r, wtmp, mixed ? rom_bl : nullptr, mixed ? rom_bc : nullptr);
        }
        RCG_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), st));
        chol_inplace(st, Ar, r, r, d_info);
        check_info("reduced matrix V^T A(p) V");
        // B~_r, C~_r: row gathers of V (point sources / receivers)
        gather_rows<T>(st, V, ld, r, c->d_rhs_node, wsrc, ns, Br, r);
        gather_rows<T>(st, V, ld, r, c->d_rhs_node + ns, wsrc + ns, nd, Crm, r);
        RCG_CUDA_TRY(cudaMemcpyAsync(Xr, Br, sizeof(double) * r * ns, cudaMemcpyDeviceToDevice, st));
        RCG_CUDA_TRY(cudaMemcpyAsync(Zr, Crm, sizeof(double) * r * nd, cudaMemcpyDeviceToDevice, st));
        trsv_lower_batched(st, Ar, r, r, Xr, r, ns, false);
        trsv_lower_batched(st, Ar, r, r, Xr, r, ns, true);
        trsv_lower_batched(st, Ar, r, r, Zr, r, nd, false);
        trsv_lower_batched(st, Ar, r, r, Zr, r, nd, true);
        // Psi_r = C~_r^T X_r  (ndet x nsrc)
        gemm_tn<double, double>(st, r, Crm, r, nd, Xr, r, ns, Psi, nd, false);
        if (J && dmu && c->track()) {
            // J_k = -Z_r^T (V^T dA~_k V) X_r + (V^T dC~_k)^T X_r + Z_r^T (V^T dB~_k): the
            // Grams of the operator derivatives (stencil and Robin terms with
            // dD = -3 D^2 dmu_k) over their rows, all J_k in one launch, then the
            // terms of the weights' derivatives from (V X_r) and (V Z_r) at the nodes
            const long long gsz = (long long)nparam * r * r;
            if (gsz > jk_gcap) {
                c->release(jk_G);
                jk_gcap = std::max(gsz, 2 * jk_gcap);
                jk_G = c->alloc<double>((size_t)jk_gcap);
            }
            RCG_CUDA_TRY(cudaMemsetAsync(jk_G, 0, sizeof(double) * (size_t)gsz, st));
            for (int k = 0; k < nparam; ++k) {
                track_deriv(st, g, tp_D, dmu + (long long)k * n, c->h, c->grid.robin_A, -1.0, tk_dg, tk_dw);
                delta_gram(V, r, jk_G + (long long)k * r * r, r);
            }
            rom_jac(st, r, nparam, jk_G, Xr, ns, Zr, nd, J);
            if (nparam > tp_dwt_cap) {
                c->release(tp_dwt);
                tp_dwt_cap = nparam;
                tp_dwt = c->alloc<double>((size_t)nparam * c->nrhs);
            }
            gather_rows<T>(st, V, ld, r, c->d_rhs_node, c->d_ones, c->nrhs, tp_G, r);   // V rows at all nodes
            double *Pd = tp_P, *Ps = tp_P + (long long)ns * nd;
            gemm_tn<double, double>(st, r, tp_G + (long long)ns * r, r, nd, Xr, r, ns, Pd, nd, false);
            gemm_tn<double, double>(st, r, tp_G, r, ns, Zr, r, nd, Ps, ns, false);
            rhs_weights(st, tp_D, c->d_rhs_node, c->d_rhs_wt, ns, c->nrhs, c->grid.robin_A, c->h, nullptr, dmu, n,
                        nparam, tp_dwt);
            jac_rhs_terms(st, nparam, nd, ns, tp_dwt, Pd, Ps, J);
        } else if (J && dmu && mixed && r >= 16 && tc_gemm_tn_ok(ld, ld, V, V)) {
            // J_k = Z_r^T G_k X_r with G_k = V^T diag(-h^2 dmu_k) V: the weighted Grams on the
            // tensor cores over the support of dmu_k (one launch for all k), then all J_k in one float64 launch
            const long long nbl = (n + 31) / 32;
            if (nparam > jk_cap) {
                for (void *p : std::vector<void *>{(void *)jk_w, (void *)jk_bl, (void *)jk_bc}) c->release(p);
                jk_cap = nparam;
                jk_w = c->alloc<double>((size_t)nparam * ld);
                jk_bl = c->alloc<int>((size_t)nparam * nbl);
                jk_bc = c->alloc<int>(nparam);
            }
            const long long gsz = (long long)nparam * r * r;
            if (gsz > jk_gcap) {
                c->release(jk_G);
                jk_gcap = std::max(gsz, 2 * jk_gcap);
                jk_G = c->alloc<double>((size_t)jk_gcap);
            }
            for (int k = 0; k < nparam; ++k)
                scaled_diff(st, n, dmu + (long long)k * n, nullptr, -c->h * c->h, jk_w + (long long)k * ld);
            tc_block_list(st, n, jk_w, jk_bl, jk_bc, nparam, ld, nbl);
            // all G_k in one tensor-core launch, then all J_k in one float64 launch
            const long long need = tc_gram_w_batched_scratch(r, nparam, nullptr);
            if (need > tc_cap) {
                c->release(tc_scr);
                tc_cap = std::max(need, 2 * tc_cap);
                tc_scr = c->alloc<float>((size_t)tc_cap);
            }
            tc_gram_w_batched(st, n, (const float *)V, ld, r, jk_G, r, (long long)r * r, nparam, jk_w, ld, jk_bl, nbl,
                              jk_bc, tc_scr, d_info + 1);
            rom_jac(st, r, nparam, jk_G, Xr, ns, Zr, nd, J);
        } else if (J && dmu) {
            if (!VX) { VX = c->alloc<double>((size_t)ns * ld); VZ = c->alloc<double>((size_t)nd * ld); }
            lift(V, r, Xr, r, ns, VX, ld, 0.0);
            lift(V, r, Zr, r, nd, VZ, ld, 0.0);
            for (int k = 0; k < nparam; ++k) {
                scaled_diff(st, n, dmu + (long long)k * n, nullptr, -c->h * c->h, wtmp);
                gemm_tn<double, double>(st, n, VZ, ld, nd, VX, ld, ns, J + (long long)k * nd * ns, nd, false, wtmp);
            }
        }
        RCG_CUDA_TRY(cudaEventRecord(e1, st));
        c->sync();
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        c->phase["rom"] = ms;
        cudaEventDestroy(e0); cudaEventDestroy(e1);
    }

    // Psi_r and J at nq points in one pass (device pointers: mu nq x n,
    // dmu nq x nparam x n or null, Psi nq x nd x ns, J nq x nparam x nd x ns):
    // the reduced matrices of all points from one tensor-core launch over the
    // supports of mu_q - mu_*, one batched Cholesky, batched solves, and, with
    // dmu, all points' Jacobian Grams in one more launch.  Where the batched
    // tensor-core path does not apply (float64 basis, r < 16, weights that
    // are not 16-byte aligned) the points run one by one through rom_eval.
    void rom_eval_batch(int nq, const double *mu, int nparam, const double *dmu, double *Psi, double *J) override {
        if (r == 0) throw Error{RCG_ERR_INVALID, "rcg_rom_eval_batch with an empty basis"};
        if (nq <= 0) return;
        const int ns = c->nsrc, nd = c->ndet;
        const bool jac = J && dmu && nparam > 0;
        const bool batched = mixed && !c->track() && r >= 16 && tc_gemm_tn_ok(ld, ld, V, V) &&
                             (!jac || ((((uintptr_t)dmu) & 15) == 0 && (n & 1) == 0));
        if (!batched) {
            for (int q = 0; q < nq; ++q)
                rom_eval(mu + (long long)q * n, jac ? nparam : 0, jac ? dmu + (long long)q * nparam * n : nullptr,
                         Psi + (long long)q * nd * ns, jac ? J + (long long)q * nparam * nd * ns : nullptr);
            return;
        }
        cudaEvent_t e0, e1;
        RCG_CUDA_TRY(cudaEventCreate(&e0)); RCG_CUDA_TRY(cudaEventCreate(&e1));
        RCG_CUDA_TRY(cudaEventRecord(e0, st));
        if (!Ar) {
            Ar = c->alloc<double>((size_t)rmax * rmax);
            Br = c->alloc<double>((size_t)rmax * ns);
            Crm = c->alloc<double>((size_t)rmax * nd);
            Xr = c->alloc<double>((size_t)rmax * ns);
            Zr = c->alloc<double>((size_t)rmax * nd);
            wtmp = c->alloc<double>(ld);
        }
        const long long nbl = (n + 31) / 32, rr2 = (long long)r * r;
        auto grow = [&](int slot, auto *&p, long long need) {
            if (need <= rb_cap[slot]) return;
            c->release(p);
            rb_cap[slot] = std::max(need, 2 * rb_cap[slot]);
            p = c->alloc<std::remove_reference_t<decltype(*p)>>((size_t)rb_cap[slot]);
        };
        grow(0, rb_A, nq * rr2);
        grow(1, rb_w, (long long)nq * ld);
        grow(2, rb_bl, nq * nbl);
        grow(3, rb_bc, (long long)nq);
        grow(4, rb_X, (long long)nq * r * ns);
        grow(5, rb_Z, (long long)nq * r * nd);
        // A~_r(q) = C_* + V^T diag(h^2 (mu_q - mu_*)) V for all q
        for (int q = 0; q < nq; ++q) {
            scaled_diff(st, n, mu + (long long)q * n, c->mu64 + (long long)s_star * ld, c->h * c->h, rb_w + (long long)q * ld);
            RCG_CUDA_TRY(cudaMemcpy2DAsync(rb_A + q * rr2, sizeof(double) * r, Cstar, sizeof(double) * rmax,
                                           sizeof(double) * r, r, cudaMemcpyDeviceToDevice, st));
        }
        tc_block_list(st, n, rb_w, rb_bl, rb_bc, nq, ld, nbl);
        const long long need = tc_gram_w_batched_scratch(r, std::max(nq, jac ? nq * nparam : 0), nullptr);
        if (need > tc_cap) {
            c->release(tc_scr);
            tc_cap = std::max(need, 2 * tc_cap);
            tc_scr = c->alloc<float>((size_t)tc_cap);
        }
        tc_gram_w_batched(st, n, (const float *)V, ld, r, rb_A, r, rr2, nq, rb_w, ld, rb_bl, nbl, rb_bc, tc_scr,
                          d_info + 1, true, 1.0);
        RCG_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), st));
        chol_batched(st, rb_A, r, rr2, r, nq, d_info);
        check_info("reduced matrices V^T A(p_q) V");
        // B~_r, C~_r (the same for every point), then X_q = A~_r(q)^-1 B~_r, Z_q likewise
        gather_rows<T>(st, V, ld, r, c->d_rhs_node, c->d_rhs_w, ns, Br, r);
        gather_rows<T>(st, V, ld, r, c->d_rhs_node + ns, c->d_rhs_w + ns, nd, Crm, r);
        for (int q = 0; q < nq; ++q) {
            RCG_CUDA_TRY(cudaMemcpyAsync(rb_X + (long long)q * r * ns, Br, sizeof(double) * r * ns,
                                         cudaMemcpyDeviceToDevice, st));
            RCG_CUDA_TRY(cudaMemcpyAsync(rb_Z + (long long)q * r * nd, Crm, sizeof(double) * r * nd,
                                         cudaMemcpyDeviceToDevice, st));
        }
        trsv_multi(st, rb_A, r, rr2, r, rb_X, r, (long long)r * ns, ns, nq, false);
        trsv_multi(st, rb_A, r, rr2, r, rb_X, r, (long long)r * ns, ns, nq, true);
        trsv_multi(st, rb_A, r, rr2, r, rb_Z, r, (long long)r * nd, nd, nq, false);
        trsv_multi(st, rb_A, r, rr2, r, rb_Z, r, (long long)r * nd, nd, nq, true);
        rom_psi(st, r, nq, Crm, rb_X, ns, nd, Psi);
        if (jac) {
            // G_qk = V^T diag(-h^2 dmu_qk) V straight from dmu (scale in the split), then J_qk = Z_q^T G_qk X_q
            const long long nv = (long long)nq * nparam;
            grow(6, rb_G, nv * rr2);
            grow(7, rb_jbl, nv * nbl);
            grow(8, rb_jbc, nv);
            tc_block_list(st, n, dmu, rb_jbl, rb_jbc, (int)nv, n, nbl);
            tc_gram_w_batched(st, n, (const float *)V, ld, r, rb_G, r, rr2, (int)nv, dmu, n, rb_jbl, nbl, rb_jbc,
                              tc_scr, d_info + 1, false, -c->h * c->h);
            rom_jac(st, r, nparam, rb_G, rb_X, ns, rb_Z, nd, J, nq);
        }
        RCG_CUDA_TRY(cudaEventRecord(e1, st));
        c->sync();
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        c->phase["rom_batch"] = ms;
        cudaEventDestroy(e0); cudaEventDestroy(e1);
    }
};

int fail(rcg_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

template <typename F> int guarded(rcg_ctx *c, F f) {
    if (!c) return RCG_ERR_INVALID;
    long long *prev = g_launch_counter;
    const long long prev_spin = g_spin_budget;
    g_launch_counter = &c->launches;
    g_spin_budget = c->opt.spin_budget;
    int rc;
    try {
        rc = f();
    } catch (const Error &e) {
        rc = fail(c, e.code, e.msg);
    } catch (const std::bad_alloc &) {
        rc = fail(c, RCG_ERR_OOM, "host allocation failed");
    } catch (...) {
        rc = fail(c, RCG_ERR_INVALID, "unexpected exception");
    }
    g_launch_counter = prev;
    g_spin_budget = prev_spin;
    return rc;
}

}  // namespace

namespace rcg {
// Operator data of a context for the allocation-free entry point (noalloc.cu).
int ctx_operator(const rcg_ctx *c, int s, Grid *g, const double **D64, const float **D32, const double **diag64,
                 const float **diag32, cudaStream_t *st, long long **launches) {
    if (!c || s < 0 || s >= c->opt.max_samples || !c->sample_set[s]) {
        if (c) const_cast<rcg_ctx *>(c)->err = "rcg_apply_noalloc: sample slot not set";
        return RCG_ERR_INVALID;
    }
    rcg_ctx *m = const_cast<rcg_ctx *>(c);
    *g = c->g;
    *D64 = c->D64;
    *D32 = c->D32;
    *diag64 = m->diag64_of(s);
    *diag32 = m->diag32_of(s);
    *st = c->st;
    *launches = &m->launches;
    return RCG_OK;
}
void ctx_set_error(rcg_ctx *c, const std::string &msg) {
    if (c) c->err = msg;
}
}  // namespace rcg

// ============================================================== C ABI
extern "C" {

void rcg_options_default(rcg_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = RCG_FP64;
    o->order = RCG_SEQUENTIAL;
    o->wave_samples = 0;
    o->tau_rank = 1e-12;
    o->k_u = 10;
    o->k_cap = 256;
    o->r_max = 2048;
    o->max_samples = 32;
    o->maxit = 20000;
    o->inner_eta = 1e-4;
    o->check_refine = -1;
    o->keep_solutions = 0;
    o->seed_degree = 0;
    o->spin_budget = 0;
    o->d_model = RCG_D_FIXED;
    o->mu_s_prime = 1.0;
}

const char *rcg_strerror(int code) {
    switch (code) {
        case RCG_OK: return "ok";
        case RCG_ERR_INVALID: return "invalid argument or call order";
        case RCG_ERR_CUDA: return "CUDA runtime error";
        case RCG_ERR_OOM: return "out of device memory";
        case RCG_ERR_NOT_SPD: return "matrix not positive definite";
        case RCG_ERR_NOT_CONVERGED: return "not converged (maximum iterations or refinement restarts reached)";
        case RCG_ERR_BREAKDOWN: return "Krylov breakdown";
        case RCG_ERR_TIMEOUT: return "device wait timed out";
        case RCG_ERR_RANK_CAP: return "basis rank cap reached";
        default: return "unknown error";
    }
}

const char *rcg_last_error(const rcg_ctx *c) { return c ? c->err.c_str() : "null context"; }

int rcg_create(rcg_ctx **out, const rcg_grid *gr, const rcg_options *o, void *stream) {
    if (!out || !gr) return RCG_ERR_INVALID;
    *out = nullptr;
    if (gr->dim != 2 && gr->dim != 3) return RCG_ERR_INVALID;
    if (gr->N < 2 || !(gr->robin_A > 0) || !std::isfinite(gr->robin_A)) return RCG_ERR_INVALID;
    if ((double)gr->N * gr->N * (gr->dim == 3 ? gr->N : 1) >= 2147483647.0) return RCG_ERR_INVALID;
    rcg_ctx *c = new (std::nothrow) rcg_ctx();
    if (!c) return RCG_ERR_OOM;
    c->grid = *gr;
    if (o) c->opt = *o; else rcg_options_default(&c->opt);
    if (c->opt.precision != RCG_FP64 && c->opt.precision != RCG_MIXED) { delete c; return RCG_ERR_INVALID; }
    if (c->opt.order != RCG_SEQUENTIAL && c->opt.order != RCG_WAVE) { delete c; return RCG_ERR_INVALID; }
    if (c->opt.wave_rhs < 0 || (c->opt.check != RCG_GALERKIN && c->opt.check != RCG_MR) ||
        (c->opt.inner != RCG_CG && c->opt.inner != RCG_MINRES) ||
        (c->opt.recycle != RCG_INNER_OUTER && c->opt.recycle != RCG_PER_RHS) ||
        // the paper's check and solver run in the float64 engine; per-RHS recycle
        // spaces hold columns outside V, which only the MINRES lanes address
        ((c->opt.check == RCG_MR || c->opt.inner == RCG_MINRES) && c->opt.precision != RCG_FP64) ||
        (c->opt.recycle == RCG_PER_RHS && c->opt.inner != RCG_MINRES) ||
        (c->opt.d_model != RCG_D_FIXED && c->opt.d_model != RCG_D_TRACKS_MU) ||
        (c->opt.learned_mode != RCG_LEARN_DEFLATE && c->opt.learned_mode != RCG_LEARN_START) ||
        (c->opt.d_model == RCG_D_TRACKS_MU && !(c->opt.mu_s_prime > 0 && std::isfinite(c->opt.mu_s_prime)))) {
        delete c;
        return RCG_ERR_INVALID;
    }
    if (c->opt.r_max < 1 || c->opt.max_samples < 1 || c->opt.k_u < 0 || c->opt.k_u > KU_MAX || c->opt.maxit < 1) {
        delete c;
        return RCG_ERR_INVALID;
    }
    if (c->opt.check_refine < 0) c->opt.check_refine = 0;
    if (!(c->opt.inner_eta > 0)) c->opt.inner_eta = 1e-4;
    c->st = (cudaStream_t)stream;
    const int N = gr->N;
    c->g.Nx = N;
    c->g.Ny = gr->dim == 3 ? N : 1;
    c->g.Nz = N;
    c->n = (long long)c->g.Nx * c->g.Ny * c->g.Nz;
    c->g.n = c->n;
    c->ld = (c->n + 63) / 64 * 64;
    c->g.ld = c->ld;
    c->h = 1.0 / (N + 1);
    c->sample_set.assign(c->opt.max_samples, 0);
    c->solutions.assign(c->opt.max_samples, {});
    int rc = guarded(c, [&]() {
        c->D64 = c->alloc<double>(c->ld);
        c->D32 = c->alloc<float>(c->ld);
        c->dstar = c->alloc<double>(c->ld);
        c->mu64 = c->alloc<double>((size_t)c->opt.max_samples * c->ld);
        c->diag64 = c->alloc<double>((size_t)c->opt.max_samples * c->ld);
        c->diag32 = c->alloc<float>((size_t)c->opt.max_samples * c->ld);
        if (c->track()) {
            // per-sample D and face weights, addressed from a sample's diagonal (Grid)
            c->Ds64 = c->alloc<double>((size_t)c->opt.max_samples * c->ld);
            c->Ds32 = c->alloc<float>((size_t)c->opt.max_samples * c->ld);
            c->Ws64 = c->alloc<double>((size_t)3 * c->opt.max_samples * c->ld);
            c->g.dbase64 = c->diag64;
            c->g.dbase32 = c->diag32;
            c->g.Ds64 = c->Ds64;
            c->g.Ds32 = c->Ds32;
            c->g.Ws64 = c->Ws64;
            c->g.dspan = (long long)c->opt.max_samples * c->ld;
        }
        c->d_prof = c->alloc<unsigned long long>(8);
        RCG_CUDA_TRY(cudaMemsetAsync(c->d_prof, 0, sizeof(unsigned long long) * 8, c->st));
        if (c->opt.precision == RCG_MIXED) c->eng.reset(new Engine<float>(c));
        else c->eng.reset(new Engine<double>(c));
        return RCG_OK;
    });
    if (rc != RCG_OK) { rcg_destroy(c); return rc; }
    *out = c;
    return RCG_OK;
}

void rcg_destroy(rcg_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->st);
    c->eng.reset();
    for (void *p : c->allocs) cudaFree(p);
    c->allocs.clear();
    delete c;
}

int rcg_set_diffusion(rcg_ctx *c, const double *D) {
    return guarded(c, [&]() {
        if (!D) return fail(c, RCG_ERR_INVALID, "D == NULL");
        for (long long p = 0; p < c->n; ++p)
            if (!(D[p] > 0) || !std::isfinite(D[p])) return fail(c, RCG_ERR_INVALID, "D must be positive and finite");
        c->h2d(c->D64, D, c->n);
        convert_cols<double, float>(c->st, c->n, c->D64, c->ld, c->D32, c->ld, 1);
        diag_star(c->st, c->g, c->D64, c->h, c->grid.robin_A, c->dstar);
        if (!c->W64) c->W64 = c->alloc<double>((size_t)3 * c->ld);
        face_weights(c->st, c->g, c->D64, c->W64);
        c->sync();
        c->have_D = true;
        c->have_rhs = false;          // effective source weights depend on D: set them again
        for (auto &s : c->sample_set) s = 0;
        return RCG_OK;
    });
}

int rcg_set_sources_detectors(rcg_ctx *c, int nsrc, const int *src_ij, const double *src_w, int ndet,
                              const int *det_ij, const double *det_w) {
    return guarded(c, [&]() {
        if (!c->have_D) return fail(c, RCG_ERR_INVALID, "rcg_set_diffusion must come first");
        if (nsrc < 0 || ndet < 0 || nsrc + ndet < 1 || (nsrc && !src_ij) || (ndet && !det_ij))
            return fail(c, RCG_ERR_INVALID, "bad source / detector lists");
        const int Nx = c->g.Nx, Ny = c->g.Ny, Nz = c->g.Nz;
        std::vector<double> Dh(c->n);
        c->d2h(Dh.data(), c->D64, c->n);
        c->sync();
        c->nsrc = nsrc;
        c->ndet = ndet;
        c->nrhs = nsrc + ndet;
        c->rhs_node.assign(c->nrhs, 0);
        c->rhs_w.assign(c->nrhs, 0.0);
        c->rhs_wt.assign(c->nrhs, 0.0);
        for (int q = 0; q < c->nrhs; ++q) {
            const bool is_src = q < nsrc;
            const int *ij = is_src ? src_ij + 2 * q : det_ij + 2 * (q - nsrc);
            const int i = ij[0], j = ij[1];
            if (i < 1 || i > Nx || j < 1 || j > Ny) return fail(c, RCG_ERR_INVALID, "face point out of range");
            const int k = is_src ? 1 : Nz;
            const long long p = (long long)(i - 1) + (long long)Nx * ((j - 1) + (long long)Ny * (k - 1));
            const double Dp = Dh[p];
            const double alpha = 2.0 * c->grid.robin_A * Dp / c->h;
            const double wt = is_src ? (src_w ? src_w[q] : 1.0) : (det_w ? det_w[q - nsrc] : 1.0);
            // b~ = s D_p / (1 + alpha_p) e_p,  c~ = c alpha_p / (1 + alpha_p) e_p  (Sec. 3.1)
            c->rhs_node[q] = (int)p;
            c->rhs_wt[q] = wt;
            c->rhs_w[q] = wt * (is_src ? Dp / (1.0 + alpha) : alpha / (1.0 + alpha));
            if (!(c->rhs_w[q] != 0.0) || !std::isfinite(c->rhs_w[q])) return fail(c, RCG_ERR_INVALID, "zero weight");
        }
        for (void *p : std::vector<void *>{c->d_rhs_node, c->d_rhs_w, c->d_rhs_wt, c->d_ones}) c->release(p);
        c->d_rhs_node = c->alloc<int>(c->nrhs);
        c->d_rhs_w = c->alloc<double>(c->nrhs);
        c->d_rhs_wt = c->alloc<double>(c->nrhs);
        c->d_ones = c->alloc<double>(c->nrhs);
        c->h2d(c->d_rhs_node, c->rhs_node.data(), c->nrhs);
        c->h2d(c->d_rhs_w, c->rhs_w.data(), c->nrhs);
        c->h2d(c->d_rhs_wt, c->rhs_wt.data(), c->nrhs);
        {
            const std::vector<double> ones((size_t)c->nrhs, 1.0);
            c->h2d(c->d_ones, ones.data(), c->nrhs);
        }
        c->tol.assign(c->nrhs, 1e-8);
        c->sync();
        c->have_rhs = true;
        return RCG_OK;
    });
}

int rcg_set_tolerances(rcg_ctx *c, const double *tol) {
    return guarded(c, [&]() {
        if (!c->have_rhs || !tol) return fail(c, RCG_ERR_INVALID, "set sources/detectors first");
        for (int j = 0; j < c->nrhs; ++j)
            if (!(tol[j] > 0 && tol[j] < 1)) return fail(c, RCG_ERR_INVALID, "tolerance out of (0, 1)");
        c->tol.assign(tol, tol + c->nrhs);
        return RCG_OK;
    });
}

static int set_sample_impl(rcg_ctx *c, int s, const double *mu, bool device) {
    return guarded(c, [&]() {
        if (!c->have_D) return fail(c, RCG_ERR_INVALID, "rcg_set_diffusion must come first");
        if (s < 0 || s >= c->opt.max_samples || !mu) return fail(c, RCG_ERR_INVALID, "bad sample slot or mu");
        double *dst = c->mu64 + (long long)s * c->ld;
        if (device) {
            RCG_CUDA_TRY(cudaMemcpyAsync(dst, mu, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->st));
        } else {
            for (long long p = 0; p < c->n; ++p)
                if (!(mu[p] >= 0) || !std::isfinite(mu[p])) return fail(c, RCG_ERR_INVALID, "mu must be >= 0 and finite");
            c->h2d(dst, mu, c->n);
        }
        if (c->track())
            track_coefficients(c->st, c->g, dst, c->opt.mu_s_prime, c->h, c->grid.robin_A, c->Ds64_of(s),
                               c->Ds32 + (long long)s * c->ld, c->Ws64_of(s), c->diag64_of(s), c->diag32_of(s));
        else
            diag_sample(c->st, c->n, c->dstar, dst, c->h * c->h, c->diag64_of(s), c->diag32_of(s));
        c->sync();
        c->sample_set[s] = 1;
        if (c->eng) c->eng->sample_changed(s);
        return RCG_OK;
    });
}

int rcg_set_sample(rcg_ctx *c, int s, const double *mu) { return set_sample_impl(c, s, mu, false); }
int rcg_set_sample_device(rcg_ctx *c, int s, const double *mu_dev) { return set_sample_impl(c, s, mu_dev, true); }

int rcg_apply_f32(rcg_ctx *c, int s, int variant, const float *x_dev, float *y_dev, int ncols, double *dots_dev) {
    return guarded(c, [&]() {
        if (s < 0 || s >= c->opt.max_samples || !c->sample_set[s] || ncols < 0 || !x_dev || !y_dev ||
            variant < -1 || variant >= RCG_STENCIL_VARIANTS)
            return fail(c, RCG_ERR_INVALID, "bad rcg_apply_f32 arguments");
        if (!cg4_supported(c->g) || ((uintptr_t)x_dev & 15) || ((uintptr_t)y_dev & 15))
            return fail(c, RCG_ERR_INVALID, "rcg_apply_f32 needs N % 4 == 0 and 16-byte aligned columns");
        if (c->track()) return fail(c, RCG_ERR_INVALID, "rcg_apply_f32: the float4 stencils take one fixed D");
        if (variant >= 0 && !stencil_variant_ok(c->g, variant))
            return fail(c, RCG_ERR_INVALID, "the stencil variant does not support this grid");
        if (ncols == 0) return RCG_OK;
        std::vector<const float *> hs(ncols), hg(ncols);
        std::vector<float *> hd(ncols);
        std::vector<int> lanes(ncols), act(ncols, 1);
        for (int j = 0; j < ncols; ++j) {
            hs[j] = x_dev + (long long)j * c->n;
            hd[j] = y_dev + (long long)j * c->n;
            hg[j] = c->diag32_of(s);
            lanes[j] = j;
        }
        const float **a = c->alloc<const float *>(ncols);
        float **b = c->alloc<float *>(ncols);
        const float **gp = c->alloc<const float *>(ncols);
        int *dl = c->alloc<int>(ncols), *da = c->alloc<int>(ncols);
        double *dd = dots_dev ? nullptr : c->alloc<double>(ncols);
        c->h2d(a, hs.data(), ncols); c->h2d(b, hd.data(), ncols); c->h2d(gp, hg.data(), ncols);
        c->h2d(dl, lanes.data(), ncols); c->h2d(da, act.data(), ncols);
        if (dd) RCG_CUDA_TRY(cudaMemsetAsync(dd, 0, sizeof(double) * ncols, c->st));
        stencil4_apply(c->st, c->g, c->D32, gp, a, b, ncols, dl, da, dots_dev ? dots_dev : dd, variant, x_dev, c->n,
                       c->diag32, c->opt.max_samples);
        c->sync();
        if (stencil_take_error(c->st)) throw Error{RCG_ERR_TIMEOUT, "rcg_apply_f32: a TMA copy's wait ran out"};
        for (void *q : std::vector<void *>{(void *)a, (void *)b, (void *)gp, (void *)dl, (void *)da, (void *)dd})
            c->release(q);
        return RCG_OK;
    });
}

const char *rcg_stencil_variant_name(int v) { return stencil_variant_name(v); }

int rcg_stencil_variant_ok(const rcg_ctx *c, int v) { return c ? stencil_variant_ok(c->g, v) : 0; }

int rcg_tuning_report(char *buf, int len) {
    try {
        const std::string r = stencil_tuning_report();
        if (buf && len > 0) {
            const int k = std::min<int>(len - 1, (int)r.size());
            std::memcpy(buf, r.data(), (size_t)k);
            buf[k] = 0;
        }
        return (int)r.size();
    } catch (...) {
        return RCG_ERR_INVALID;
    }
}

int rcg_apply(rcg_ctx *c, int s, int prec, const void *x_dev, void *y_dev, int ncols) {
    return guarded(c, [&]() {
        if (s < 0 || s >= c->opt.max_samples || !c->sample_set[s] || ncols < 0 || !x_dev || !y_dev)
            return fail(c, RCG_ERR_INVALID, "bad rcg_apply arguments");
        if (prec == RCG_FP64) {
            std::vector<const double *> hs(ncols), hg(ncols);
            std::vector<double *> hd(ncols);
            for (int j = 0; j < ncols; ++j) {
                hs[j] = (const double *)x_dev + (long long)j * c->n;
                hd[j] = (double *)y_dev + (long long)j * c->n;
                hg[j] = c->diag64_of(s);
            }
            const double **a = c->alloc<const double *>(ncols);
            double **b = c->alloc<double *>(ncols);
            const double **g = c->alloc<const double *>(ncols);
            c->h2d(a, hs.data(), ncols); c->h2d(b, hd.data(), ncols); c->h2d(g, hg.data(), ncols);
            apply_op<double>(c->st, c->g, c->D64, g, a, b, ncols, nullptr, nullptr);
            c->sync();
            c->release((void *)a); c->release(b); c->release((void *)g);
        } else if (prec == RCG_MIXED) {
            std::vector<const float *> hs(ncols), hg(ncols);
            std::vector<float *> hd(ncols);
            for (int j = 0; j < ncols; ++j) {
                hs[j] = (const float *)x_dev + (long long)j * c->n;
                hd[j] = (float *)y_dev + (long long)j * c->n;
                hg[j] = c->diag32_of(s);
            }
            const float **a = c->alloc<const float *>(ncols);
            float **b = c->alloc<float *>(ncols);
            const float **g = c->alloc<const float *>(ncols);
            c->h2d(a, hs.data(), ncols); c->h2d(b, hd.data(), ncols); c->h2d(g, hg.data(), ncols);
            apply_op<float>(c->st, c->g, c->D32, g, a, b, ncols, nullptr, nullptr);
            c->sync();
            c->release((void *)a); c->release(b); c->release((void *)g);
        } else {
            return fail(c, RCG_ERR_INVALID, "prec must be RCG_FP64 or RCG_MIXED");
        }
        return RCG_OK;
    });
}

int rcg_seed(rcg_ctx *c, int s0, const double *U0, rcg_stat *stats) {
    return guarded(c, [&]() {
        if (!c->have_rhs || s0 < 0 || s0 >= c->opt.max_samples || !c->sample_set[s0])
            return fail(c, RCG_ERR_INVALID, "rcg_seed needs D, sources/detectors and sample s0");
        c->eng->seed(s0, U0, stats);
        return RCG_OK;
    });
}

int rcg_seed_copy(rcg_ctx *c, const rcg_ctx *src) {
    return guarded(c, [&]() {
        if (!src || src == c || !src->eng || !c->eng) return fail(c, RCG_ERR_INVALID, "rcg_seed_copy: bad contexts");
        if (c->grid.dim != src->grid.dim || c->grid.N != src->grid.N || c->grid.robin_A != src->grid.robin_A ||
            c->rhs_node != src->rhs_node || c->rhs_w != src->rhs_w || !c->have_D || !src->have_D ||
            c->opt.d_model != src->opt.d_model || (c->track() && c->opt.mu_s_prime != src->opt.mu_s_prime))
            return fail(c, RCG_ERR_INVALID, "rcg_seed_copy: grid, sources / detectors or D model differ");
        const SeedView sv = src->eng->seed_view();
        if (!sv.seeded) return fail(c, RCG_ERR_INVALID, "rcg_seed_copy: the source context is not seeded");
        if (sv.s_star < 0 || sv.s_star >= c->opt.max_samples || !c->sample_set[sv.s_star])
            return fail(c, RCG_ERR_INVALID, "rcg_seed_copy: set the seed sample slot first");
        // D and the seed sample's mu must be the ones the seed was built for
        const size_t n = (size_t)c->n;
        std::vector<double> a(n), b(n);
        c->d2h(a.data(), c->D64, n);
        c->sync();
        RCG_CUDA_TRY(cudaMemcpy(b.data(), src->D64, sizeof(double) * n, cudaMemcpyDeviceToHost));
        bool same = a == b;
        c->d2h(a.data(), c->mu64 + (long long)sv.s_star * c->ld, n);
        c->sync();
        RCG_CUDA_TRY(cudaMemcpy(b.data(), src->mu64 + (long long)sv.s_star * src->ld, sizeof(double) * n,
                                cudaMemcpyDeviceToHost));
        same = same && a == b;
        if (!same) return fail(c, RCG_ERR_INVALID, "rcg_seed_copy: D or the seed sample's mu differ");
        c->eng->seed_import(sv);
        return RCG_OK;
    });
}

int rcg_reset_to_seed(rcg_ctx *c) {
    return guarded(c, [&]() { c->eng->reset(); return RCG_OK; });
}

int rcg_solve_all(rcg_ctx *c, int s_first, int s_count, rcg_stat *stats) {
    return guarded(c, [&]() {
        if (s_first < 0 || s_count < 1 || s_first + s_count > c->opt.max_samples)
            return fail(c, RCG_ERR_INVALID, "bad sample range");
        for (int s = s_first; s < s_first + s_count; ++s)
            if (!c->sample_set[s]) return fail(c, RCG_ERR_INVALID, "sample not set");
        const int rc = c->eng->solve_all(s_first, s_count, stats);
        if (rc != RCG_OK) c->err = rcg_strerror(rc);
        return rc;
    });
}

int rcg_basis_rank(const rcg_ctx *c, int *r) {
    if (!c || !r) return RCG_ERR_INVALID;
    *r = c->eng->rank();
    return RCG_OK;
}

int rcg_basis_get(rcg_ctx *c, double *V) {
    return guarded(c, [&]() {
        if (!V) return fail(c, RCG_ERR_INVALID, "V == NULL");
        c->eng->basis_get(V);
        return RCG_OK;
    });
}

int rcg_solution_get(rcg_ctx *c, int s, double *X) {
    return guarded(c, [&]() {
        if (!c->opt.keep_solutions || s < 0 || s >= c->opt.max_samples || !X || c->solutions[s].empty())
            return fail(c, RCG_ERR_INVALID, "no kept solutions for this sample");
        std::memcpy(X, c->solutions[s].data(), sizeof(double) * c->solutions[s].size());
        return RCG_OK;
    });
}

// rcg_full_eval with D tracking mu at sample s: the weights at D_s and
//   J_k = -Z^T dA~_k X + dC~_k^T X + Z^T dB~_k
// (dA~_k: the operator derivative with dD = -3 D_s^2 dmu_k, applied on its
// rows; dB~_k, dC~_k: the weights' derivatives at the source / detector nodes).
static int full_eval_tracking(rcg_ctx *c, int s, int nparam, const double *dmu, double *Psi, double *J) {
    const int ns = c->nsrc, nd = c->ndet, nrhs = c->nrhs;
    const long long n = c->n, ld = c->ld;
    const std::vector<double> &X = c->solutions[s];
    std::vector<double> ws(nrhs);
    double *d_ws = c->alloc<double>(nrhs);
    rhs_weights(c->st, c->Ds64_of(s), c->d_rhs_node, c->d_rhs_wt, ns, nrhs, c->grid.robin_A, c->h, d_ws);
    c->d2h(ws.data(), d_ws, nrhs);
    c->sync();
    c->release(d_ws);
    for (int j = 0; j < ns; ++j)
        for (int d = 0; d < nd; ++d)
            Psi[d + (long long)nd * j] = ws[ns + d] * X[(size_t)j * n + c->rhs_node[ns + d]];
    if (!dmu) return RCG_OK;
    const long long nbl = (n + 31) / 32;
    double *dX = c->alloc<double>((size_t)nrhs * ld), *dm = c->alloc<double>((size_t)nparam * n);
    double *dg = c->alloc<double>(ld), *dw = c->alloc<double>((size_t)3 * ld), *touch = c->alloc<double>(ld);
    double *dJ = c->alloc<double>((size_t)nparam * nd * ns), *dwt = c->alloc<double>((size_t)nparam * nrhs);
    int *bl = c->alloc<int>((size_t)nbl), *bc = c->alloc<int>(1);
    double *Xc = c->alloc<double>((size_t)nbl * 32 * nrhs), *Yc = c->alloc<double>((size_t)nbl * 32 * nrhs);
    for (int j = 0; j < nrhs; ++j) c->h2d(dX + (long long)j * ld, X.data() + (size_t)j * n, (size_t)n);
    c->h2d(dm, dmu, (size_t)nparam * n);
    for (int k = 0; k < nparam; ++k) {
        double *Jk = dJ + (long long)k * nd * ns;
        track_deriv(c->st, c->g, c->Ds64_of(s), dm + (long long)k * n, c->h, c->grid.robin_A, -1.0, dg, dw);
        track_touch(c->st, c->g, dg, dw, touch);
        tc_block_list(c->st, n, touch, bl, bc);
        int nb = 0;
        c->d2h(&nb, bc, 1);
        c->sync();
        if (nb <= 0) {
            RCG_CUDA_TRY(cudaMemsetAsync(Jk, 0, sizeof(double) * (size_t)nd * ns, c->st));
            continue;
        }
        const long long rows = (long long)nb * 32;
        // -Z^T dA_k X over the rows of dA_k: Z rows (detector columns of Xc) against dA_k X
        delta_rows<double>(c->st, c->g, bl, 0, nb, dg, dw, dX, ld, nrhs, Xc, Yc, rows);
        gemm_tn<double, double>(c->st, rows, Xc + (long long)ns * rows, rows, nd, Yc, rows, ns, Jk, nd, false);
    }
    rhs_weights(c->st, c->Ds64_of(s), c->d_rhs_node, c->d_rhs_wt, ns, nrhs, c->grid.robin_A, c->h, nullptr, dm, n,
                nparam, dwt);
    std::vector<double> hdwt((size_t)nparam * nrhs);
    c->d2h(J, dJ, (size_t)nparam * nd * ns);
    c->d2h(hdwt.data(), dwt, hdwt.size());
    c->sync();
    for (void *p : std::vector<void *>{dX, dm, dg, dw, touch, dJ, dwt, bl, bc, Xc, Yc}) c->release(p);
    // the weights' terms: dC~_k^T x_j = dc_{k,d} x_j(node_d), z_d^T dB~_k = db_{k,j} z_d(node_j)
    for (int k = 0; k < nparam; ++k)
        for (int j = 0; j < ns; ++j)
            for (int d = 0; d < nd; ++d)
                J[(long long)k * nd * ns + d + (long long)nd * j] +=
                    hdwt[(size_t)k * nrhs + ns + d] * X[(size_t)j * n + c->rhs_node[ns + d]] +
                    hdwt[(size_t)k * nrhs + j] * X[(size_t)(ns + d) * n + c->rhs_node[j]];
    return RCG_OK;
}

int rcg_full_eval(rcg_ctx *c, int s, int nparam, const double *dmu, double *Psi, double *J) {
    return guarded(c, [&]() {
        if (!c->opt.keep_solutions || s < 0 || s >= c->opt.max_samples || !Psi || c->solutions[s].empty())
            return fail(c, RCG_ERR_INVALID, "rcg_full_eval: no kept solutions for this sample");
        if (dmu && (nparam < 1 || !J)) return fail(c, RCG_ERR_INVALID, "rcg_full_eval: nparam / J");
        const int ns = c->nsrc, nd = c->ndet;
        const long long n = c->n, ld = c->ld;
        const std::vector<double> &X = c->solutions[s];       // n x nrhs, sources then detectors
        if (c->track()) return full_eval_tracking(c, s, nparam, dmu, Psi, J);
        // Psi[d, j] = c~_d^T x_j: the receivers are point functionals w_d e_{node_d}
        for (int j = 0; j < ns; ++j)
            for (int d = 0; d < nd; ++d)
                Psi[d + (long long)nd * j] = c->rhs_w[ns + d] * X[(size_t)j * n + c->rhs_node[ns + d]];
        if (dmu) {
            double *dX = c->alloc<double>((size_t)c->nrhs * ld), *dw = c->alloc<double>((size_t)ld);
            double *dm = c->alloc<double>((size_t)ld), *dJ = c->alloc<double>((size_t)nparam * nd * ns);
            for (int j = 0; j < c->nrhs; ++j) c->h2d(dX + (long long)j * ld, X.data() + (size_t)j * n, (size_t)n);
            for (int k = 0; k < nparam; ++k) {
                c->h2d(dm, dmu + (size_t)k * n, (size_t)n);
                scaled_diff(c->st, n, dm, nullptr, -c->h * c->h, dw);
                gemm_tn<double, double>(c->st, n, dX + (long long)ns * ld, ld, nd, dX, ld, ns,
                                        dJ + (long long)k * nd * ns, nd, false, dw);
            }
            c->d2h(J, dJ, (size_t)nparam * nd * ns);
            c->sync();
            for (void *p : std::vector<void *>{dX, dw, dm, dJ}) c->release(p);
        }
        return RCG_OK;
    });
}

int rcg_save(rcg_ctx *c, const char *path) {
    return guarded(c, [&]() {
        if (!path || !c->eng) return fail(c, RCG_ERR_INVALID, "rcg_save: no path or nothing to save");
        std::FILE *f = std::fopen(path, "wb");
        if (!f) return fail(c, RCG_ERR_INVALID, std::string("rcg_save: cannot open ") + path);
        try {
            wr(f, kMagic, sizeof(kMagic));
            long long mus_bits = 0;
            std::memcpy(&mus_bits, &c->opt.mu_s_prime, sizeof(mus_bits));
            const long long g[8] = {c->grid.dim, c->grid.N, c->n, c->opt.precision, c->nsrc, c->ndet,
                                    c->opt.d_model, c->track() ? mus_bits : 0};
            wr(f, g, sizeof(g));
            std::vector<double> D((size_t)c->n);
            c->d2h(D.data(), c->D64, (size_t)c->n);
            c->sync();
            wr_vec(f, D);
            wr_vec(f, c->rhs_node);
            wr_vec(f, c->rhs_w);
            c->eng->save(f);
            const bool have_net = c->cnn && c->cnn->have;
            const long long nn = have_net ? c->cnn->P : 0;
            wr(f, &nn, sizeof(nn));
            if (have_net) {
                std::vector<float> th((size_t)nn);
                c->d2h(th.data(), c->cnn->theta, (size_t)nn);
                c->sync();
                wr(f, th.data(), sizeof(float) * th.size());
            }
        } catch (...) {
            std::fclose(f);
            throw;
        }
        if (std::fclose(f) != 0) return fail(c, RCG_ERR_INVALID, "rcg_save: close failed");
        return RCG_OK;
    });
}

int rcg_load(rcg_ctx *c, const char *path) {
    return guarded(c, [&]() {
        if (!path) return fail(c, RCG_ERR_INVALID, "rcg_load: no path");
        if (!c->have_D || !c->have_rhs) return fail(c, RCG_ERR_INVALID, "rcg_load: set D and the sources first");
        std::FILE *f = std::fopen(path, "rb");
        if (!f) return fail(c, RCG_ERR_INVALID, std::string("rcg_load: cannot open ") + path);
        try {
            char m[8];
            rd(f, m, sizeof(m));
            if (std::memcmp(m, kMagic, sizeof(m)) != 0) throw Error{RCG_ERR_INVALID, "rcg_load: not an rcg state file"};
            long long g[8];
            rd(f, g, sizeof(g));
            long long mus_bits = 0;
            std::memcpy(&mus_bits, &c->opt.mu_s_prime, sizeof(mus_bits));
            if (g[0] != c->grid.dim || g[1] != c->grid.N || g[2] != c->n || g[3] != c->opt.precision ||
                g[4] != c->nsrc || g[5] != c->ndet || g[6] != c->opt.d_model || g[7] != (c->track() ? mus_bits : 0))
                throw Error{RCG_ERR_INVALID, "rcg_load: grid, precision, source/detector counts or D model differ"};
            auto D = rd_vec<double>(f, c->n);
            auto node = rd_vec<int>(f, c->nrhs);
            auto w = rd_vec<double>(f, c->nrhs);
            std::vector<double> Dc((size_t)c->n);
            c->d2h(Dc.data(), c->D64, (size_t)c->n);
            c->sync();
            if (D != Dc || node != c->rhs_node || w != c->rhs_w)
                throw Error{RCG_ERR_INVALID, "rcg_load: D or the sources / detectors differ from the saved state"};
            if (!c->eng) throw Error{RCG_ERR_INVALID, "rcg_load: context has no engine"};
            c->eng->load(f);
            long long nn = 0;
            rd(f, &nn, sizeof(nn));
            if (nn) {
                if (nn != cnn_nparams()) throw Error{RCG_ERR_INVALID, "rcg_load: network size differs"};
                std::vector<float> th((size_t)nn);
                rd(f, th.data(), sizeof(float) * th.size());
                c->net().set_weights(c->st, th.data());
                c->sync();
            }
        } catch (...) {
            std::fclose(f);
            throw;
        }
        std::fclose(f);
        return RCG_OK;
    });
}

int rcg_rom_eval_device(rcg_ctx *c, const double *mu_dev, int nparam, const double *dmu_dev, double *Psi_dev,
                        double *J_dev) {
    return guarded(c, [&]() {
        if (!mu_dev || !Psi_dev || nparam < 0) return fail(c, RCG_ERR_INVALID, "bad rom arguments");
        c->eng->rom_eval(mu_dev, nparam, dmu_dev, Psi_dev, J_dev);
        return RCG_OK;
    });
}

int rcg_basis_compress(rcg_ctx *c, int r_max, double tau, double *sigma, int sigma_len, int *nsnap) {
    return guarded(c, [&]() {
        if (!(tau >= 0.0) || sigma_len < 0 || (sigma_len > 0 && !sigma))
            return fail(c, RCG_ERR_INVALID, "bad compress arguments");
        std::vector<double> sg;
        const int m = c->eng->compress(r_max, tau, sg);
        for (int i = 0; i < std::min(sigma_len, m); ++i) sigma[i] = sg[i];
        if (nsnap) *nsnap = m;
        return RCG_OK;
    });
}

int rcg_rom_eval_batch_chunk(long long n, int r, int nsrc, int ndet, int nparam) {
    if (n < 0 || r < 0 || nsrc < 0 || ndet < 0 || nparam < 0) return -1;
    const long long ld = (n + 63) / 64 * 64, nbl = (n + 31) / 32, rr = (long long)r * r;
    long long per = 8 * rr + 8 * ld + 4 * nbl + 4 + 8LL * r * (nsrc + ndet);
    if (nparam > 0) per += (long long)nparam * (8 * rr + 4 * nbl + 4);
    for (int k = 256; k > 1; --k) {
        // the tensor-core partial sums of the chunk's weight vectors (k reduced
        // matrices, then k nparam Jacobian Grams, in one scratch buffer)
        const long long scr = rcg::tc_gram_w_batched_scratch(std::max(r, 1), k * std::max(nparam, 1), nullptr);
        if (k * per + 4 * scr <= RCG_ROM_BATCH_WORKSPACE) return k;
    }
    return 1;
}

int rcg_rom_eval_batch(rcg_ctx *c, int nq, const double *mu_dev, int nparam, const double *dmu_dev,
                       double *Psi_dev, double *J_dev) {
    return guarded(c, [&]() {
        if (nq < 0 || nparam < 0 || (nq > 0 && (!mu_dev || !Psi_dev)) || (J_dev && !dmu_dev))
            return fail(c, RCG_ERR_INVALID, "bad rom batch arguments");
        // chunks of points: bounded workspace (per point r x r matrices and n weights,
        // per point and parameter a Gram) and grid dimensions
        const int CHUNK = std::max(1, rcg_rom_eval_batch_chunk(c->n, c->eng->rank(), c->nsrc, c->ndet,
                                                               J_dev ? nparam : 0));
        const long long n = c->n, nd_ns = (long long)c->ndet * c->nsrc;
        for (int q0 = 0; q0 < nq; q0 += CHUNK) {
            const int m = std::min(CHUNK, nq - q0);
            c->eng->rom_eval_batch(m, mu_dev + (long long)q0 * n, nparam,
                                   dmu_dev ? dmu_dev + (long long)q0 * nparam * n : nullptr, Psi_dev + q0 * nd_ns,
                                   J_dev ? J_dev + (long long)q0 * nparam * nd_ns : nullptr);
        }
        return RCG_OK;
    });
}

int rcg_rom_eval(rcg_ctx *c, const double *mu, int nparam, const double *dmu, double *Psi, double *J) {
    return guarded(c, [&]() {
        if (!mu || !Psi || nparam < 0 || (J && !dmu)) return fail(c, RCG_ERR_INVALID, "bad rom arguments");
        const long long n = c->n;
        double *dmu_d = nullptr, *mu_d = c->alloc<double>(n);
        double *P = c->alloc<double>((size_t)c->nsrc * c->ndet);
        double *Jd = nullptr;
        c->h2d(mu_d, mu, n);
        if (J) {
            dmu_d = c->alloc<double>((size_t)n * std::max(nparam, 1));
            Jd = c->alloc<double>((size_t)c->nsrc * c->ndet * std::max(nparam, 1));
            c->h2d(dmu_d, dmu, (size_t)n * nparam);
        }
        c->eng->rom_eval(mu_d, nparam, dmu_d, P, Jd);
        c->d2h(Psi, P, (size_t)c->nsrc * c->ndet);
        if (J) c->d2h(J, Jd, (size_t)c->nsrc * c->ndet * nparam);
        c->sync();
        c->release(mu_d); c->release(P); c->release(dmu_d); c->release(Jd);
        return RCG_OK;
    });
}

double rcg_phase_ms(const rcg_ctx *c, const char *phase) {
    if (!c || !phase) return -1.0;
    auto it = c->phase.find(phase);
    return it == c->phase.end() ? -1.0 : it->second;
}

long long rcg_launch_count(const rcg_ctx *c) { return c ? c->launches : -1; }

// ------------------------------------------------------------ learned
int rcg_learn_nparams(void) { return cnn_nparams(); }

int rcg_learn_geometry(rcg_ctx *c, int *dims) {
    return guarded(c, [&]() {
        if (!dims) throw Error{RCG_ERR_INVALID, "rcg_learn_geometry: dims is NULL"};
        const CnnGeom cg = cnn_geom(c->g);
        dims[0] = cg.Gx; dims[1] = cg.Gy; dims[2] = cg.Gz; dims[3] = cg.f;
        return RCG_OK;
    });
}

int rcg_learn_set_weights(rcg_ctx *c, const float *theta, int nparam) {
    return guarded(c, [&]() {
        if (!theta || nparam != cnn_nparams()) throw Error{RCG_ERR_INVALID, "rcg_learn_set_weights: nparam mismatch"};
        for (int i = 0; i < nparam; ++i)
            if (!std::isfinite(theta[i])) throw Error{RCG_ERR_INVALID, "rcg_learn_set_weights: non-finite weight"};
        c->net().set_weights(c->st, theta);
        c->sync();
        return RCG_OK;
    });
}

int rcg_learn_get_weights(rcg_ctx *c, float *theta, int nparam) {
    return guarded(c, [&]() {
        if (!theta || nparam != cnn_nparams()) throw Error{RCG_ERR_INVALID, "rcg_learn_get_weights: nparam mismatch"};
        if (!c->cnn || !c->cnn->have) throw Error{RCG_ERR_INVALID, "rcg_learn_get_weights: no weights yet"};
        c->d2h(theta, c->cnn->theta, nparam);
        c->sync();
        return RCG_OK;
    });
}

int rcg_learn_record(rcg_ctx *c, int on) {
    return guarded(c, [&]() {
        if (c->opt.precision != RCG_MIXED) throw Error{RCG_ERR_INVALID, "rcg_learn_record: RCG_MIXED only"};
        c->net().record = on != 0;
        return RCG_OK;
    });
}

int rcg_learn_pairs(rcg_ctx *c, int *npairs) {
    return guarded(c, [&]() {
        if (!npairs) throw Error{RCG_ERR_INVALID, "rcg_learn_pairs: NULL"};
        *npairs = c->cnn ? c->cnn->npairs : 0;
        return RCG_OK;
    });
}

int rcg_learn_train(rcg_ctx *c, int epochs, int batch, double lr, unsigned long long seed, double *loss) {
    return guarded(c, [&]() {
        if (epochs < 0 || batch < 1 || !(lr > 0.0)) throw Error{RCG_ERR_INVALID, "rcg_learn_train: bad arguments"};
        if (!c->cnn || !c->cnn->have) throw Error{RCG_ERR_INVALID, "rcg_learn_train: set initial weights first"};
        const double l = c->cnn->train(c->st, epochs, batch, lr, seed);
        if (loss) *loss = l;
        return RCG_OK;
    });
}

int rcg_learn_forward(rcg_ctx *c, const float *in, int B, float *out) {
    return guarded(c, [&]() {
        if (!in || !out || B < 1) throw Error{RCG_ERR_INVALID, "rcg_learn_forward: bad arguments"};
        Cnn &net = c->net();
        if (!net.have) throw Error{RCG_ERR_INVALID, "rcg_learn_forward: no weights"};
        const long long V = net.geom.V;
        float *din = c->alloc<float>((size_t)B * 2 * V), *dout = c->alloc<float>((size_t)B * V);
        c->h2d(din, in, (size_t)B * 2 * V);
        net.forward(c->st, din, B, dout);
        c->d2h(out, dout, (size_t)B * V);
        c->sync();
        c->release(din);
        c->release(dout);
        return RCG_OK;
    });
}

int rcg_learn_gradient(rcg_ctx *c, const float *in, const float *tg, int B, float *grad, double *loss) {
    return guarded(c, [&]() {
        if (!in || !tg || !grad || B < 1) throw Error{RCG_ERR_INVALID, "rcg_learn_gradient: bad arguments"};
        Cnn &net = c->net();
        if (!net.have) throw Error{RCG_ERR_INVALID, "rcg_learn_gradient: no weights"};
        const long long V = net.geom.V;
        float *din = c->alloc<float>((size_t)B * 2 * V), *dtg = c->alloc<float>((size_t)B * V);
        c->h2d(din, in, (size_t)B * 2 * V);
        c->h2d(dtg, tg, (size_t)B * V);
        const double l = net.gradient(c->st, din, dtg, B);
        c->d2h(grad, net.grad, net.P);
        c->sync();
        c->release(din);
        c->release(dtg);
        if (loss) *loss = l;
        return RCG_OK;
    });
}

int rcg_learn_predict(rcg_ctx *c, int s, const float *r0, float *feat, float *xhat) {
    return guarded(c, [&]() {
        if (!r0 || s < 0 || s >= c->opt.max_samples || !c->sample_set[s])
            throw Error{RCG_ERR_INVALID, "rcg_learn_predict: bad arguments or sample slot not set"};
        Cnn &net = c->net();
        if (!net.have) throw Error{RCG_ERR_INVALID, "rcg_learn_predict: no weights"};
        const long long V = net.geom.V;
        float *dr = c->alloc<float>((size_t)c->ld), *df = c->alloc<float>((size_t)2 * V), *dout = c->alloc<float>(V);
        float *dx = c->alloc<float>((size_t)c->ld);
        const float **pr = c->alloc<const float *>(1);
        const double **pm = c->alloc<const double *>(1);
        float **px = c->alloc<float *>(1);
        const float *hr = dr;
        const double *hm = c->mu64 + (long long)s * c->ld;
        float *hx = dx;
        c->h2d(dr, r0, (size_t)c->n);
        c->h2d(pr, &hr, 1);
        c->h2d(pm, &hm, 1);
        c->h2d(px, &hx, 1);
        net.features(c->st, pr, pm, 1, df);
        net.forward(c->st, df, 1, dout);
        net.upsample(c->st, dout, px, nullptr, 1);
        if (feat) c->d2h(feat, df, (size_t)2 * V);
        if (xhat) c->d2h(xhat, dx, (size_t)c->n);
        c->sync();
        for (void *p : std::vector<void *>{dr, df, dout, dx, (void *)pr, (void *)pm, (void *)px}) c->release(p);
        return RCG_OK;
    });
}

int rcg_profile_enable(rcg_ctx *c, int on) {
    return guarded(c, [&]() {
        c->sync();
        c->ktimer.reset();
        c->ktimer.on = on != 0;
        RCG_CUDA_TRY(cudaMemsetAsync(c->d_prof, 0, sizeof(unsigned long long) * 8, c->st));
        c->sync();
        return RCG_OK;
    });
}

int rcg_profile_get(rcg_ctx *c, int kernel, rcg_kprof *out) {
    return guarded(c, [&]() {
        if (!out || kernel < 0 || kernel >= KTimer::NK) return fail(c, RCG_ERR_INVALID, "bad profile query");
        c->sync();
        c->ktimer.harvest();
        unsigned long long h[8];
        c->d2h(h, c->d_prof, 8);
        c->sync();
        out->launches = c->ktimer.launches[kernel];
        out->ms = c->ktimer.ms[kernel];
        // stencil: column applications; update: lanes; the other three: direction lanes
        out->lane_units = (double)(kernel == 0 ? h[0] : kernel == 1 ? h[1] : h[3]);
        out->defl_cols = (double)(kernel == 0 ? 0 : kernel == 1 ? h[2] : h[4]);
        return RCG_OK;
    });
}

}  // extern "C"
