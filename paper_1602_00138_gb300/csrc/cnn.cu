// Learned augmentation of the private recycle space (not in the paper; the
// build's learned step): a coarse-grid 3D CNN that maps a right-hand side's
// Galerkin-check residual r0 and the sample's absorption mu to the shape of
// the correction g = A~^-1 r0 that the inner deflated CG (eq. resi) solves
// for.  Its upsampled output joins the private deflation space of that solve.
//
//   features   block means over f^3 fine nodes: [coarse(r0) / max|coarse(r0)|,
//              coarse(mu) / mean(mu) - 1], rounded to bfloat16
//   network    a 3-level U-Net (16-32-64 channels, ten 3x3x3 convolutions,
//              skip connections) on the coarse grid, bfloat16 activations and
//              weights on the tensor cores with float32 accumulation
//              (unet.cu); training keeps float32 master weights (Adam, mean
//              squared error against coarse(g) / max|coarse(g)|) and computes
//              the gradient with bfloat16 operands
//   upsample   trilinear interpolation from coarse cell centres to fine nodes
//
// Parameter layout: per layer W [Cout][Cin][27] (offset (dz+1)*9+(dy+1)*3+(dx+1))
// then b [Cout].  Activations are [batch][channel][coarse node], x fastest.
#include "common.cuh"
#include "../../include/rcg.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <numeric>
#include <random>

namespace rcg {

namespace {

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void coords(long long v, int Gx, int Gy, int &x, int &y, int &z) {
    x = (int)(v % Gx);
    const long long t = v / Gx;
    y = (int)(t % Gy);
    z = (int)(t / Gy);
}

// Block means of r0 (float32) and mu (float64) of lane blockIdx.x, then the
// normalisation of both channels and the bfloat16 rounding.
__global__ void __launch_bounds__(256)
k_cnn_features(CnnGeom cg, const float *const *__restrict__ r0, const double *const *__restrict__ mu,
               float *__restrict__ out) {
    const int l = blockIdx.x;
    const float *__restrict__ r = r0[l];
    const double *__restrict__ m = mu[l];
    float *o0 = out + (long long)l * 2 * cg.V, *o1 = o0 + cg.V;
    const int fy = cg.Ny > 1 ? cg.f : 1;
    const float inv = 1.0f / (float)(cg.f * fy * cg.f);
    float amax = 0.f, msum = 0.f;
    for (long long v = threadIdx.x; v < cg.V; v += blockDim.x) {
        int cx, cy, cz;
        coords(v, cg.Gx, cg.Gy, cx, cy, cz);
        float sr = 0.f, sm = 0.f;
        for (int dz = 0; dz < cg.f; ++dz)
            for (int dy = 0; dy < fy; ++dy) {
                const long long base =
                    ((long long)(cz * cg.f + dz) * cg.Ny + (cy * fy + dy)) * cg.Nx + (long long)cx * cg.f;
                for (int dx = 0; dx < cg.f; ++dx) {
                    sr += r[base + dx];
                    sm += (float)m[base + dx];
                }
            }
        sr *= inv;
        sm *= inv;
        o0[v] = sr;
        o1[v] = sm;
        amax = fmaxf(amax, fabsf(sr));
        msum += sm;
    }
    __shared__ float s_max[8], s_sum[8];
    for (int o = 16; o > 0; o >>= 1) {
        amax = fmaxf(amax, __shfl_down_sync(0xffffffffu, amax, o));
        msum += __shfl_down_sync(0xffffffffu, msum, o);
    }
    if ((threadIdx.x & 31) == 0) { s_max[threadIdx.x >> 5] = amax; s_sum[threadIdx.x >> 5] = msum; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a = fmaxf(a, s_max[w]); s += s_sum[w]; }
        s_max[0] = a;
        s_sum[0] = s / (float)cg.V;
    }
    __syncthreads();
    const float a = s_max[0], mean = s_sum[0];
    const float ia = a > 0.f ? 1.0f / a : 1.0f;
    for (long long v = threadIdx.x; v < cg.V; v += blockDim.x) {
        o0[v] = bf16_round(o0[v] * ia);
        o1[v] = bf16_round(o1[v] / mean - 1.0f);
    }
}

// dout = 2 (out - t) / (B V); loss += sum (out - t)^2 / (B V)
__global__ void k_mse(const float *__restrict__ out, const float *__restrict__ t, float *__restrict__ dout,
                      long long tot, double *__restrict__ loss) {
    float s = 0.f;
    const float sc = 1.0f / (float)tot;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const float d = out[e] - t[e];
        dout[e] = 2.f * d * sc;
        s += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, (double)s / (double)tot);
}

__global__ void k_adam(float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int P, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_round_bf16(const float *__restrict__ a, float *__restrict__ b, int P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) b[i] = bf16_round(a[i]);
}

__global__ void k_gather_pairs(const float *__restrict__ src, long long stride, const int *__restrict__ idx, int B,
                               float *__restrict__ dst) {
    const int b = blockIdx.y;
    const float *s = src + (long long)idx[b] * stride;
    float *d = dst + (long long)b * stride;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < stride; e += (long long)gridDim.x * blockDim.x)
        d[e] = s[e];
}

// Trilinear interpolation of coarse row rows[b] (b if rows is NULL) to the
// fine column dst[b].
__global__ void k_cnn_upsample(CnnGeom cg, const float *__restrict__ out, float *const *__restrict__ dst,
                               const int *__restrict__ rows) {
    const int b = blockIdx.y;
    const float *__restrict__ c = out + (long long)(rows ? rows[b] : b) * cg.V;
    float *__restrict__ y = dst[b];
    const long long n = (long long)cg.Nx * cg.Ny * cg.Nz;
    const int fy = cg.Ny > 1 ? cg.f : 1;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % cg.Nx);
        const long long t = p / cg.Nx;
        const int yy = (int)(t % cg.Ny), z = (int)(t / cg.Ny);
        auto axis = [](int i, int f, int G, int &i0, int &i1, float &w) {
            const float tt = ((float)i + 0.5f) / (float)f - 0.5f;
            const int fl = (int)floorf(tt);
            w = tt - (float)fl;
            i0 = min(max(fl, 0), G - 1);
            i1 = min(max(fl + 1, 0), G - 1);
        };
        int x0, x1, y0, y1, z0, z1;
        float wx, wy, wz;
        axis(x, cg.f, cg.Gx, x0, x1, wx);
        axis(yy, fy, cg.Gy, y0, y1, wy);
        axis(z, cg.f, cg.Gz, z0, z1, wz);
        auto at = [&](int a, int bb, int cc) { return c[((long long)cc * cg.Gy + bb) * cg.Gx + a]; };
        const float c00 = at(x0, y0, z0) * (1.f - wx) + at(x1, y0, z0) * wx;
        const float c10 = at(x0, y1, z0) * (1.f - wx) + at(x1, y1, z0) * wx;
        const float c01 = at(x0, y0, z1) * (1.f - wx) + at(x1, y0, z1) * wx;
        const float c11 = at(x0, y1, z1) * (1.f - wx) + at(x1, y1, z1) * wx;
        const float c0 = c00 * (1.f - wy) + c10 * wy, c1 = c01 * (1.f - wy) + c11 * wy;
        y[p] = c0 * (1.f - wz) + c1 * wz;
    }
}

// Coarse means of a float64 column (for the training target, on x0 and x).
__global__ void k_cnn_pool64(CnnGeom cg, const double *const *__restrict__ src, float *__restrict__ out, float sign,
                             int accumulate) {
    const int l = blockIdx.y;
    const double *__restrict__ s = src[l];
    const int fy = cg.Ny > 1 ? cg.f : 1;
    const float inv = 1.0f / (float)(cg.f * fy * cg.f);
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < cg.V; v += (long long)gridDim.x * blockDim.x) {
        int cx, cy, cz;
        coords(v, cg.Gx, cg.Gy, cx, cy, cz);
        double acc = 0.0;
        for (int dz = 0; dz < cg.f; ++dz)
            for (int dy = 0; dy < fy; ++dy) {
                const long long base =
                    ((long long)(cz * cg.f + dz) * cg.Ny + (cy * fy + dy)) * cg.Nx + (long long)cx * cg.f;
                for (int dx = 0; dx < cg.f; ++dx) acc += s[base + dx];
            }
        const float val = sign * (float)acc * inv;
        float *o = out + (long long)l * cg.V + v;
        *o = accumulate ? *o + val : val;
    }
}

// Normalise each row of [B][V] by its max |.| (training targets).
__global__ void __launch_bounds__(256) k_cnn_normalise(float *__restrict__ a, long long V) {
    float *r = a + (long long)blockIdx.x * V;
    float m = 0.f;
    for (long long v = threadIdx.x; v < V; v += blockDim.x) m = fmaxf(m, fabsf(r[v]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    __shared__ float s[8];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, s[w]);
        s[0] = t;
    }
    __syncthreads();
    const float im = s[0] > 0.f ? 1.0f / s[0] : 1.0f;
    for (long long v = threadIdx.x; v < V; v += blockDim.x) r[v] *= im;
}

// cd[a][q] += (A~ x_hat)^T w_q over this CTA's nodes for augmented lane
// l = alist[a]: w_q = U_0 column q (q < ku), private column q - ku (q < ku + kp),
// and x_hat itself (q = ku + kp, the slot the network's column occupies).
__global__ void __launch_bounds__(256)
k_aug_dots(long long n, long long ld, const float *__restrict__ V, int ku, const float *const *__restrict__ wpp,
           const float *__restrict__ awp, int kps, const int *__restrict__ kp, const int *__restrict__ alist,
           double *__restrict__ cd, long long chunk) {
    constexpr int NQ = KU_MAX + KP_MAX + 1;
    __shared__ const float *cols[NQ];
    const int a = blockIdx.y, l = alist[a];
    const int kpl = kp[l], nq = ku + kpl + 1;
    if (threadIdx.x < NQ) {
        const int q = threadIdx.x;
        cols[q] = q < ku ? V + (long long)q * ld : q < nq ? wpp[(long long)l * KPT + (q - ku)] : nullptr;
    }
    __syncthreads();
    const float *__restrict__ y = awp + ((long long)l * kps + kpl) * ld;
    // chunk is a multiple of 4 and every column starts 16-byte aligned: float4
    // loads up to the last full group of four, scalar loads for a ragged end
    const long long r0 = (long long)blockIdx.x * chunk, r1 = min(r0 + chunk, n);
    const long long r4 = r0 + ((r1 - r0) & ~3LL);
    float acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.f;
    for (long long p = r0 + 4 * (long long)threadIdx.x; p < r4; p += 4 * (long long)blockDim.x) {
        const float4 yv = *(const float4 *)(y + p);
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (q < nq) {
                const float4 w = *(const float4 *)(cols[q] + p);
                acc[q] = fmaf(yv.x, w.x, fmaf(yv.y, w.y, fmaf(yv.z, w.z, fmaf(yv.w, w.w, acc[q]))));
            }
    }
    for (long long p = r4 + threadIdx.x; p < r1; p += blockDim.x) {
        const float yv = y[p];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (q < nq) acc[q] += yv * cols[q][p];
    }
    __shared__ float red[8][NQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        float v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
        atomicAdd(cd + (long long)a * (KMAX + 1) + threadIdx.x, (double)v);
    }
}

// Galerkin pivot of x_hat against U_j: s = d - c^T G^-1 c (G^-1 in gw, c the
// first k entries of cd, d the last).  Kept iff d > 0 and sqrt(s / d) > tau;
// then G^-1 is bordered by the block-inverse formula and kdef, kp grow by one.
__global__ void __launch_bounds__(64)
k_aug_border(double *__restrict__ gw, int *__restrict__ kdef, int *__restrict__ kp, const int *__restrict__ alist,
             const double *__restrict__ cd, double tau, int *__restrict__ kept) {
    const int a = blockIdx.x, l = alist[a];
    const int k = kdef[l];
    double *G = gw + (long long)l * KMAX * KMAX;
    const double *c = cd + (long long)a * (KMAX + 1);
    const double d = c[k];
    __shared__ double t[KMAX];
    __shared__ double s_s;
    __shared__ int s_keep;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double v = 0.0;
        for (int j = 0; j < k; ++j) v += G[i + j * KMAX] * c[j];
        t[i] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ctc = 0.0;
        for (int i = 0; i < k; ++i) ctc += c[i] * t[i];
        const double sv = d - ctc;
        const bool keep = k < KMAX && d > 0.0 && sv > 0.0 && isfinite(sv) && sqrt(sv / d) > tau;
        s_s = sv;
        s_keep = keep ? 1 : 0;
        kept[a] = s_keep;
    }
    __syncthreads();
    if (!s_keep) return;
    const double is = 1.0 / s_s;
    for (int e = threadIdx.x; e < (k + 1) * (k + 1); e += blockDim.x) {
        const int i = e % (k + 1), j = e / (k + 1);
        double v;
        if (i < k && j < k) v = G[i + j * KMAX] + t[i] * t[j] * is;
        else if (i < k) v = -t[i] * is;
        else if (j < k) v = -t[j] * is;
        else v = is;
        G[i + j * KMAX] = v;      // in place: entry (i, j) is read (i, j < k) and written by this thread only
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        kdef[l] = k + 1;
        kp[l] = kp[l] + 1;
    }
}

template <typename K>
void set_smem(K kern, size_t bytes) {
    if (bytes > 48 * 1024) RCG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

}  // namespace

// ------------------------------------------------------------------ geometry
CnnGeom cnn_geom(const Grid &g) {
    CnnGeom cg{};
    cg.Nx = g.Nx; cg.Ny = g.Ny; cg.Nz = g.Nz;
    auto ok = [&](int f) { return g.Nx % f == 0 && g.Nz % f == 0 && (g.Ny == 1 || g.Ny % f == 0); };
    cg.f = ok(4) ? 4 : ok(2) ? 2 : 1;
    cg.Gx = g.Nx / cg.f;
    cg.Gy = g.Ny > 1 ? g.Ny / cg.f : 1;
    cg.Gz = g.Nz / cg.f;
    cg.V = (long long)cg.Gx * cg.Gy * cg.Gz;
    return cg;
}

int cnn_nparams() {
    int P = 0;
    for (int l = 0; l < UNET_LAYERS; ++l) P += UNET_COUT[l] * UNET_CIN[l] * 27 + UNET_COUT[l];
    return P;
}

// ------------------------------------------------------------------ network
Cnn::Cnn(const Grid &g) : geom(cnn_geom(g)), P(cnn_nparams()), net(geom.Gx, geom.Gy, geom.Gz) {
    if (net.P != P) throw Error{RCG_ERR_INVALID, "learned network: parameter layouts disagree"};
    RCG_CUDA_TRY(cudaMalloc(&theta, sizeof(float) * P));
    RCG_CUDA_TRY(cudaMalloc(&theta16, sizeof(float) * P));
    RCG_CUDA_TRY(cudaMalloc(&grad, sizeof(float) * P));
    RCG_CUDA_TRY(cudaMalloc(&adam_m, sizeof(float) * P));
    RCG_CUDA_TRY(cudaMalloc(&adam_v, sizeof(float) * P));
    RCG_CUDA_TRY(cudaMalloc(&d_loss, sizeof(double)));
}

Cnn::~Cnn() {
    for (void *p : std::vector<void *>{theta, theta16, grad, adam_m, adam_v, d_loss, act, pin, ptg, bin, btg, d_idx,
                                       feat, outc, x0c})
        if (p) cudaFree(p);
}

void Cnn::ensure(float *&p, long long &cap, long long need) {
    if (need <= cap) return;
    if (p) RCG_CUDA_TRY(cudaFree(p));
    p = nullptr;
    cap = 0;
    RCG_CUDA_TRY(cudaMalloc(&p, sizeof(float) * (size_t)need));
    cap = need;
}

void Cnn::set_weights(cudaStream_t st, const float *host) {
    RCG_CUDA_TRY(cudaMemcpyAsync(theta, host, sizeof(float) * P, cudaMemcpyHostToDevice, st));
    RCG_CUDA_TRY(cudaMemsetAsync(adam_m, 0, sizeof(float) * P, st));
    RCG_CUDA_TRY(cudaMemsetAsync(adam_v, 0, sizeof(float) * P, st));
    t_adam = 0;
    refresh_bf16(st);
    have = true;
}

// bfloat16 copy of the master weights (inference biases) and the packed
// bfloat16 weights of the tensor-core convolutions
void Cnn::refresh_bf16(cudaStream_t st) {
    k_round_bf16<<<(P + 255) / 256, 256, 0, st>>>(theta, theta16, P);
    count_launch();
    RCG_CHECK_LAUNCH();
    net.pack(st, theta, false);
}

void Cnn::features(cudaStream_t st, const float *const *r0, const double *const *mu, int nl, float *out) {
    if (nl <= 0) return;
    k_cnn_features<<<nl, 256, 0, st>>>(geom, r0, mu, out);
    count_launch();
    RCG_CHECK_LAUNCH();
}

// Inference on B inputs [B][2][V] -> out [B][V] with the bfloat16 weights,
// in chunks of items whose activations fit in about 2 GB.
void Cnn::forward(cudaStream_t st, const float *in, int B, float *out) {
    const long long V = geom.V;
    const int chunk = (int)std::max<long long>(1, std::min<long long>(B, (2LL << 30) / net.bytes_per_item()));
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int nb = std::min(chunk, B - b0);
        net.forward(st, theta16, in + (long long)b0 * 2 * V, nb, out + (long long)b0 * V);
    }
    if (net.error(st)) throw Error{RCG_ERR_TIMEOUT, "learned network: a tensor-core wait ran out"};
}

// One training batch: the forward pass with the master weights rounded to
// bfloat16 (master biases), the mean squared error and its gradient, the
// backward pass into `grad`; the loss is accumulated into d_loss.
void Cnn::forward_backward(cudaStream_t st, const float *in, const float *tg, int B) {
    const long long V = geom.V;
    ensure(act, act_cap, 2LL * B * V);
    float *outp = act, *dout = act + (long long)B * V;
    net.pack(st, theta, true);
    net.forward(st, theta, in, B, outp);
    k_mse<<<(int)std::min<long long>((B * V + 255) / 256, 1024), 256, 0, st>>>(outp, tg, dout, (long long)B * V, d_loss);
    count_launch();
    RCG_CHECK_LAUNCH();
    net.backward(st, dout, B, grad);
}

double Cnn::gradient(cudaStream_t st, const float *in, const float *tg, int B) {
    RCG_CUDA_TRY(cudaMemsetAsync(d_loss, 0, sizeof(double), st));
    forward_backward(st, in, tg, B);
    double h = 0.0;
    RCG_CUDA_TRY(cudaMemcpyAsync(&h, d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    RCG_CUDA_TRY(cudaStreamSynchronize(st));
    if (net.error(st)) throw Error{RCG_ERR_TIMEOUT, "learned network: a tensor-core wait ran out"};
    return h;
}

// Pairs recorded from solves: features [2][V] and target [V] each.
void Cnn::add_pairs(cudaStream_t st, const float *feat, const float *tgt, int cnt) {
    if (cnt <= 0) return;
    const long long V = geom.V;
    long long need = (long long)(npairs + cnt);
    if (need > pair_cap) {
        long long cap = std::max(need, 2 * pair_cap);
        float *a = nullptr, *b = nullptr;
        RCG_CUDA_TRY(cudaMalloc(&a, sizeof(float) * (size_t)cap * 2 * V));
        RCG_CUDA_TRY(cudaMalloc(&b, sizeof(float) * (size_t)cap * V));
        if (npairs) {
            RCG_CUDA_TRY(cudaMemcpyAsync(a, pin, sizeof(float) * (size_t)npairs * 2 * V, cudaMemcpyDeviceToDevice, st));
            RCG_CUDA_TRY(cudaMemcpyAsync(b, ptg, sizeof(float) * (size_t)npairs * V, cudaMemcpyDeviceToDevice, st));
            RCG_CUDA_TRY(cudaStreamSynchronize(st));
        }
        if (pin) cudaFree(pin);
        if (ptg) cudaFree(ptg);
        pin = a;
        ptg = b;
        pair_cap = cap;
    }
    RCG_CUDA_TRY(cudaMemcpyAsync(pin + (long long)npairs * 2 * V, feat, sizeof(float) * (size_t)cnt * 2 * V,
                                 cudaMemcpyDeviceToDevice, st));
    RCG_CUDA_TRY(cudaMemcpyAsync(ptg + (long long)npairs * V, tgt, sizeof(float) * (size_t)cnt * V,
                                 cudaMemcpyDeviceToDevice, st));
    npairs += cnt;
}

// Adam over the recorded pairs: `epochs` passes in shuffled batches of B.
double Cnn::train(cudaStream_t st, int epochs, int B, double lr, unsigned long long seed) {
    if (npairs <= 0) throw Error{RCG_ERR_INVALID, "rcg_learn_train: no recorded pairs"};
    const long long V = geom.V;
    B = std::max(1, std::min(B, npairs));
    ensure(bin, bin_cap, (long long)B * 2 * V);
    ensure(btg, btg_cap, (long long)B * V);
    if (idx_cap < npairs) {
        if (d_idx) cudaFree(d_idx);
        d_idx = nullptr;
        RCG_CUDA_TRY(cudaMalloc(&d_idx, sizeof(int) * (size_t)npairs));
        idx_cap = npairs;
    }
    std::mt19937_64 rng(seed);
    std::vector<int> order(npairs);
    std::iota(order.begin(), order.end(), 0);
    double last = 0.0;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(order.begin(), order.end(), rng);
        // pageable source: the copy has left `order` when the call returns
        RCG_CUDA_TRY(cudaMemcpyAsync(d_idx, order.data(), sizeof(int) * (size_t)npairs, cudaMemcpyHostToDevice, st));
        RCG_CUDA_TRY(cudaMemsetAsync(d_loss, 0, sizeof(double), st));
        int nb = 0;
        for (int b0 = 0; b0 + B <= npairs; b0 += B) {       // whole batches only
            k_gather_pairs<<<dim3(64, B), 256, 0, st>>>(pin, 2 * V, d_idx + b0, B, bin);
            count_launch();
            RCG_CHECK_LAUNCH();
            k_gather_pairs<<<dim3(32, B), 256, 0, st>>>(ptg, V, d_idx + b0, B, btg);
            count_launch();
            RCG_CHECK_LAUNCH();
            forward_backward(st, bin, btg, B);
            ++t_adam;
            const float c1 = 1.f - powf(b1, (float)t_adam), c2 = 1.f - powf(b2, (float)t_adam);
            k_adam<<<(P + 255) / 256, 256, 0, st>>>(theta, grad, adam_m, adam_v, P, (float)lr, b1, b2, eps, c1, c2);
            count_launch();
            RCG_CHECK_LAUNCH();
            ++nb;
        }
        double h = 0.0;
        RCG_CUDA_TRY(cudaMemcpyAsync(&h, d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        RCG_CUDA_TRY(cudaStreamSynchronize(st));
        last = nb ? h / nb : 0.0;
    }
    if (net.error(st)) throw Error{RCG_ERR_TIMEOUT, "learned network: a tensor-core wait ran out"};
    refresh_bf16(st);
    have = true;
    return last;
}

void Cnn::upsample(cudaStream_t st, const float *out, float *const *dst, const int *rows, int B) {
    if (B <= 0) return;
    const long long n = (long long)geom.Nx * geom.Ny * geom.Nz;
    dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 1024), (unsigned)B);
    k_cnn_upsample<<<grid, 256, 0, st>>>(geom, out, dst, rows);
    count_launch();
    RCG_CHECK_LAUNCH();
}

// targets: coarse(x) - coarse(x0), normalised; x0c holds coarse(x0) of the lanes
void Cnn::pool64(cudaStream_t st, const double *const *src, float *out, int B, float sign, bool accumulate) {
    if (B <= 0) return;
    dim3 grid((unsigned)std::min<long long>((geom.V + 255) / 256, 256), (unsigned)B);
    k_cnn_pool64<<<grid, 256, 0, st>>>(geom, src, out, sign, accumulate ? 1 : 0);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void Cnn::normalise(cudaStream_t st, float *a, int B) {
    if (B <= 0) return;
    k_cnn_normalise<<<B, 256, 0, st>>>(a, geom.V);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void aug_dots(cudaStream_t st, long long n, long long ld, const float *V, int ku, const float *const *wpp,
              const float *awp, int kps, const int *kp, const int *alist, int na, double *cd) {
    if (na <= 0) return;
    RCG_CUDA_TRY(cudaMemsetAsync(cd, 0, sizeof(double) * (size_t)na * (KMAX + 1), st));
    // chunks of ~8192 nodes (a multiple of 4): thousands of CTAs over the lanes
    long long z = std::max<long long>(1, (n + 8191) / 8192);
    long long chunk = (n + z - 1) / z;
    chunk = (chunk + 3) / 4 * 4;
    z = (n + chunk - 1) / chunk;
    if (ld % 4 != 0) throw Error{RCG_ERR_INVALID, "aug_dots: leading dimension not a multiple of 4"};
    k_aug_dots<<<dim3((unsigned)z, (unsigned)na), 256, 0, st>>>(n, ld, V, ku, wpp, awp, kps, kp, alist, cd, chunk);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void aug_border(cudaStream_t st, double *gw, int *kdef, int *kp, const int *alist, int na, const double *cd,
                double tau, int *kept) {
    if (na <= 0) return;
    k_aug_border<<<na, 64, 0, st>>>(gw, kdef, kp, alist, cd, tau, kept);
    count_launch();
    RCG_CHECK_LAUNCH();
}

}  // namespace rcg
