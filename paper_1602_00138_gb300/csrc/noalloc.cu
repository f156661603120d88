// rcg_apply_noalloc: the operator application of rcg_apply without any
// device allocation.  rcg_apply builds three device tables (source column,
// destination column and diagonal pointer of every column) in memory it
// allocates and frees on each call; this variant keeps the tables in one
// file-scope static device array instead, so that callers whose device
// memory is owned by another allocator, or that must not pay for
// cudaMalloc / cudaFree (cudaFree waits for the device) in a repeated
// call, can still apply the operator.  The caller passes x and y.
//
// The array holds tables for at most RCG_NOALLOC_MAX_COLS columns; every GPU
// that loads the library keeps it until the process exits.  All calls share
// it and it keeps the last call's tables, so calls that overlap on the GPU
// (different streams, or different host threads) race on it.
#include "common.cuh"
#include "../../include/rcg.h"

#include <mutex>
#include <new>
#include <string>
#include <vector>

namespace {

constexpr int kMaxCols = RCG_NOALLOC_MAX_COLS;

// [0, kMaxCols): source columns, [kMaxCols, 2 kMaxCols): destination columns,
// [2 kMaxCols, 3 kMaxCols): diagonal of each column.
static __device__ __align__(256) const void *g_noalloc_tables[3 * kMaxCols];

std::mutex g_mu;
void *g_addr[64] = {nullptr};   // device address of g_noalloc_tables, per device ordinal

// Resolve the device address of the static array on the current device
// (once per device).  Host code must not use g_noalloc_tables directly: on
// the host that name is only a stand-in, not a device address.
int tables_address(void **out, std::string &err) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        err = "cudaGetDevice failed";
        return RCG_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_tables);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return RCG_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return RCG_OK;
}

}  // namespace

namespace rcg {
// Operator data of a context needed here (defined in api.cu).
int ctx_operator(const rcg_ctx *c, int s, Grid *g, const double **D64, const float **D32, const double **diag64,
                 const float **diag32, cudaStream_t *st, long long **launches);
void ctx_set_error(rcg_ctx *c, const std::string &msg);
}  // namespace rcg

namespace {
int apply_noalloc(rcg_ctx *c, int s, int prec, const void *x_dev, void *y_dev, int ncols) {
    using namespace rcg;
    if (!c) return RCG_ERR_INVALID;
    if (ncols < 0 || ncols > kMaxCols || !x_dev || !y_dev || (prec != RCG_FP64 && prec != RCG_MIXED)) {
        ctx_set_error(c, "rcg_apply_noalloc: ncols must be in [0, " + std::to_string(kMaxCols) +
                             "], x and y non-null, prec RCG_FP64 or RCG_MIXED");
        return RCG_ERR_INVALID;
    }
    Grid g{};
    const double *D64 = nullptr, *diag64 = nullptr;
    const float *D32 = nullptr, *diag32 = nullptr;
    cudaStream_t st = nullptr;
    long long *launches = nullptr;
    int rc = ctx_operator(c, s, &g, &D64, &D32, &diag64, &diag32, &st, &launches);
    if (rc != RCG_OK) return rc;
    if (ncols == 0) return RCG_OK;
    void *tab = nullptr;
    std::string err;
    rc = tables_address(&tab, err);
    if (rc != RCG_OK) {
        ctx_set_error(c, err);
        return rc;
    }
    const size_t es = prec == RCG_FP64 ? sizeof(double) : sizeof(float);
    long long *prev = g_launch_counter;
    g_launch_counter = launches;
    rc = RCG_OK;
    try {
        // the three tables of this call (ncols entries each) in one host buffer
        std::vector<const void *> h(3 * (size_t)ncols, nullptr);
        for (int j = 0; j < ncols; ++j) {
            h[j] = (const char *)x_dev + (size_t)j * g.n * es;
            h[(size_t)ncols + j] = (char *)y_dev + (size_t)j * g.n * es;
            h[2 * (size_t)ncols + j] = prec == RCG_FP64 ? (const void *)diag64 : (const void *)diag32;
        }
        const void **t = (const void **)tab;
        for (int part = 0; part < 3; ++part)     // only the entries in use, into their table of the array
            RCG_CUDA_TRY(cudaMemcpyAsync(t + (size_t)part * kMaxCols, h.data() + (size_t)part * ncols,
                                         sizeof(void *) * (size_t)ncols, cudaMemcpyHostToDevice, st));
        if (prec == RCG_FP64)
            apply_op<double>(st, g, D64, (const double *const *)(t + 2 * kMaxCols), (const double *const *)t,
                             (double *const *)(t + kMaxCols), ncols, nullptr, nullptr);
        else
            apply_op<float>(st, g, D32, (const float *const *)(t + 2 * kMaxCols), (const float *const *)t,
                            (float *const *)(t + kMaxCols), ncols, nullptr, nullptr);
        // the host table h is pageable and goes out of scope: wait for the copies and the kernel
        RCG_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (const Error &e) {
        ctx_set_error(c, e.msg);
        rc = e.code;
    } catch (const std::bad_alloc &) {
        ctx_set_error(c, "rcg_apply_noalloc: host allocation failed");
        rc = RCG_ERR_OOM;
    } catch (...) {
        ctx_set_error(c, "rcg_apply_noalloc: unexpected exception");
        rc = RCG_ERR_INVALID;
    }
    g_launch_counter = prev;
    return rc;
}
}  // namespace

extern "C" int rcg_apply_noalloc(rcg_ctx *c, int s, int prec, const void *x_dev, void *y_dev, int ncols) {
    // no C++ exception may cross the C boundary (the error messages are
    // std::strings and can throw on the host)
    try {
        return apply_noalloc(c, s, prec, x_dev, y_dev, ncols);
    } catch (const std::bad_alloc &) {
        return RCG_ERR_OOM;
    } catch (...) {
        return RCG_ERR_INVALID;
    }
}
