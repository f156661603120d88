// Learned augmentation of the private recycle space (not in the paper; the
// build's learned step): a coarse-grid 3D CNN that maps a right-hand side's
// Galerkin-check residual r0 and the sample's absorption mu to the shape of
// the correction g = A~^-1 r0 that the inner deflated CG (eq. resi) solves
// for.  Its upsampled output joins the private deflation space of that solve.
//
//   features   block means over f^3 fine nodes: [coarse(r0) / max|coarse(r0)|,
//              coarse(mu) / mean(mu) - 1], rounded to bfloat16
//   network    channels 2 -> 16 -> 16 -> 16 -> 16 -> 16 -> 1, 3x3x3 zero-padded
//              convolutions with bias, ReLU between layers; inference uses the
//              bfloat16-rounded weights (products of bfloat16 values, float32
//              sums), training the float32 master weights (Adam, mean squared
//              error against coarse(g) / max|coarse(g)|)
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

const int CNN_CH[CNN_LAYERS + 1] = {2, 16, 16, 16, 16, 16, 1};

namespace {

constexpr int CT = 128;          // threads of the convolution kernels
constexpr int CMAX = 16;         // widest layer

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

// out[b][co][p] = bias[co] + sum_ci sum_d W[co][ci][d] in[b][ci][p + d]  (zero
// padding), optional ReLU.  One thread per VX consecutive x nodes (Gx % VX ==
// 0), all COUT outputs; the weights sit in shared memory as [ci][27][COUT] so
// that a (ci, d) step reads them as float4 broadcasts and uses each for VX nodes.
template <int COUT, int VX>
__global__ void __launch_bounds__(CT)
k_conv3_fwd(const float *__restrict__ in, int Cin, float *__restrict__ out, const float *__restrict__ W,
            const float *__restrict__ bias, int relu, int Gx, int Gy, int Gz, long long V) {
    extern __shared__ float4 wsm4[];
    float *wsm = (float *)wsm4;
    for (int e = threadIdx.x; e < COUT * Cin * 27; e += CT) {
        const int co = e / (Cin * 27), rem = e % (Cin * 27);       // rem = ci*27 + d
        wsm[rem * COUT + co] = W[e];
    }
    __syncthreads();
    const long long v0 = ((long long)blockIdx.x * CT + threadIdx.x) * VX;
    if (v0 >= V) return;
    const int b = blockIdx.y;
    int x, y, z;
    coords(v0, Gx, Gy, x, y, z);
    float acc[VX][COUT];
#pragma unroll
    for (int j = 0; j < VX; ++j)
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[j][co] = bias[co];
    for (int ci = 0; ci < Cin; ++ci) {
        const float *__restrict__ src = in + ((long long)b * Cin + ci) * V;
        for (int dzy = 0; dzy < 9; ++dzy) {
            const int yy = y + dzy % 3 - 1, zz = z + dzy / 3 - 1;
            if (yy < 0 || yy >= Gy || zz < 0 || zz >= Gz) continue;
            const float *row = src + ((long long)zz * Gy + yy) * Gx;
            // x - 1 .. x + VX: the row segment every tap of this (dz, dy) needs
            float seg[VX + 2];
#pragma unroll
            for (int j = 0; j < VX + 2; ++j) {
                const int xx = x + j - 1;
                seg[j] = (xx >= 0 && xx < Gx) ? row[xx] : 0.f;
            }
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const float *w = wsm + (ci * 27 + dzy * 3 + dx) * COUT;
                if constexpr (COUT % 4 == 0) {
#pragma unroll
                    for (int q = 0; q < COUT / 4; ++q) {
                        const float4 w4 = ((const float4 *)w)[q];
#pragma unroll
                        for (int j = 0; j < VX; ++j) {
                            const float val = seg[j + dx];
                            acc[j][4 * q] += w4.x * val;
                            acc[j][4 * q + 1] += w4.y * val;
                            acc[j][4 * q + 2] += w4.z * val;
                            acc[j][4 * q + 3] += w4.w * val;
                        }
                    }
                } else {
#pragma unroll
                    for (int co = 0; co < COUT; ++co)
#pragma unroll
                        for (int j = 0; j < VX; ++j) acc[j][co] += w[co] * seg[j + dx];
                }
            }
        }
    }
#pragma unroll
    for (int co = 0; co < COUT; ++co)
#pragma unroll
        for (int j = 0; j < VX; ++j) {
            float a = acc[j][co];
            if (relu) a = fmaxf(a, 0.f);
            out[((long long)b * COUT + co) * V + v0 + j] = a;
        }
}

// din[b][ci][q] = (sum_co sum_d W[co][ci][d] dout[b][co][q - d]) * (act[b][ci][q] > 0):
// the gradient with respect to the input of a layer whose input is a ReLU output.
template <int CIN>
__global__ void __launch_bounds__(CT)
k_conv3_bwd_data(const float *__restrict__ dout, int Cout, const float *__restrict__ W,
                 const float *__restrict__ act, float *__restrict__ din, int Gx, int Gy, int Gz, long long V) {
    extern __shared__ float4 wsm4[];
    float *wsm = (float *)wsm4;
    for (int e = threadIdx.x; e < Cout * CIN * 27; e += CT) {
        const int co = e / (CIN * 27), rem = e % (CIN * 27), ci = rem / 27, d = rem % 27;
        wsm[(co * 27 + d) * CIN + ci] = W[e];
    }
    __syncthreads();
    const long long v = (long long)blockIdx.x * CT + threadIdx.x;
    if (v >= V) return;
    const int b = blockIdx.y;
    int x, y, z;
    coords(v, Gx, Gy, x, y, z);
    float acc[CIN];
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.f;
    for (int co = 0; co < Cout; ++co) {
        const float *__restrict__ src = dout + ((long long)b * Cout + co) * V;
        for (int d = 0; d < 27; ++d) {
            // input node v feeds output node v - d
            const int xx = x - (d % 3 - 1), yy = y - ((d / 3) % 3 - 1), zz = z - (d / 9 - 1);
            if (xx < 0 || xx >= Gx || yy < 0 || yy >= Gy || zz < 0 || zz >= Gz) continue;
            const float g = src[((long long)zz * Gy + yy) * Gx + xx];
            const float4 *w4 = (const float4 *)(wsm + (co * 27 + d) * CIN);
#pragma unroll
            for (int q = 0; q < CIN / 4; ++q) {
                const float4 w = w4[q];
                acc[4 * q] += w.x * g;
                acc[4 * q + 1] += w.y * g;
                acc[4 * q + 2] += w.z * g;
                acc[4 * q + 3] += w.w * g;
            }
        }
    }
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) {
        const long long o = ((long long)b * CIN + ci) * V + v;
        din[o] = act[o] > 0.f ? acc[ci] : 0.f;
    }
}

// dW[co][ci][d] = sum_b sum_p dout[b][co][p] in[b][ci][p + d]; db[co] = sum dout.
// One CTA per (co, ci) pair; 27 sums per thread, reduced in shared memory.
__global__ void __launch_bounds__(256)
k_conv3_bwd_w(const float *__restrict__ dout, int Cout, const float *__restrict__ in, int Cin,
              float *__restrict__ dW, float *__restrict__ db, int B, int Gx, int Gy, int Gz, long long V) {
    const int co = blockIdx.x / Cin, ci = blockIdx.x % Cin;
    float acc[27], ab = 0.f;
#pragma unroll
    for (int d = 0; d < 27; ++d) acc[d] = 0.f;
    const long long tot = (long long)B * V;
    for (long long e = threadIdx.x; e < tot; e += blockDim.x) {
        const int b = (int)(e / V);
        const long long v = e % V;
        int x, y, z;
        coords(v, Gx, Gy, x, y, z);
        const float g = dout[((long long)b * Cout + co) * V + v];
        ab += g;
        const float *__restrict__ src = in + ((long long)b * Cin + ci) * V;
#pragma unroll
        for (int d = 0; d < 27; ++d) {
            const int xx = x + d % 3 - 1, yy = y + (d / 3) % 3 - 1, zz = z + d / 9 - 1;
            if (xx >= 0 && xx < Gx && yy >= 0 && yy < Gy && zz >= 0 && zz < Gz)
                acc[d] += g * src[((long long)zz * Gy + yy) * Gx + xx];
        }
    }
    __shared__ float red[8][28];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 28; ++d) {
        float s = d < 27 ? acc[d] : ab;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp][d] = s;
    }
    __syncthreads();
    if (threadIdx.x < 28) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        if (threadIdx.x < 27) dW[((long long)co * Cin + ci) * 27 + threadIdx.x] = s;
        else if (ci == 0) db[co] = s;
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
    for (int l = 0; l < CNN_LAYERS; ++l) P += CNN_CH[l + 1] * CNN_CH[l] * 27 + CNN_CH[l + 1];
    return P;
}

// ------------------------------------------------------------------ network
Cnn::Cnn(const Grid &g) : geom(cnn_geom(g)), P(cnn_nparams()) {
    RCG_CUDA_TRY(cudaMalloc(&theta, sizeof(float) * P));
    RCG_CUDA_TRY(cudaMalloc(&theta16, sizeof(float) * P));
    RCG_CUDA_TRY(cudaMalloc(&grad, sizeof(float) * P));
    RCG_CUDA_TRY(cudaMalloc(&adam_m, sizeof(float) * P));
    RCG_CUDA_TRY(cudaMalloc(&adam_v, sizeof(float) * P));
    RCG_CUDA_TRY(cudaMalloc(&d_loss, sizeof(double)));
    int o = 0;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        woff[l] = o;
        o += CNN_CH[l + 1] * CNN_CH[l] * 27;
        boff[l] = o;
        o += CNN_CH[l + 1];
    }
}

Cnn::~Cnn() {
    for (void *p : std::vector<void *>{theta, theta16, grad, adam_m, adam_v, d_loss, act, dact0, dact1, pin, ptg,
                                       bin, btg, d_idx, feat, outc, x0c})
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

void Cnn::refresh_bf16(cudaStream_t st) {
    k_round_bf16<<<(P + 255) / 256, 256, 0, st>>>(theta, theta16, P);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void Cnn::features(cudaStream_t st, const float *const *r0, const double *const *mu, int nl, float *out) {
    if (nl <= 0) return;
    k_cnn_features<<<nl, 256, 0, st>>>(geom, r0, mu, out);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void Cnn::conv(cudaStream_t st, int l, const float *in, float *out, int B, bool relu, bool rounded) {
    const int Cin = CNN_CH[l], Cout = CNN_CH[l + 1];
    const float *Wt = (rounded ? theta16 : theta) + woff[l];
    const float *bt = (rounded ? theta16 : theta) + boff[l];
    const size_t sm = sizeof(float) * (size_t)Cout * Cin * 27;
    const int vx = geom.Gx % 4 == 0 ? 4 : 1;
    const long long thr = (geom.V + vx - 1) / vx;
    dim3 grid((unsigned)((thr + CT - 1) / CT), (unsigned)B);
#define RCG_CONV(CO, VXT) k_conv3_fwd<CO, VXT><<<grid, CT, sm, st>>>(in, Cin, out, Wt, bt, relu ? 1 : 0, geom.Gx, \
                                                                     geom.Gy, geom.Gz, geom.V)
    if (Cout == 16) {
        if (vx == 4) RCG_CONV(16, 4);
        else RCG_CONV(16, 1);
    } else {
        if (vx == 4) RCG_CONV(1, 4);
        else RCG_CONV(1, 1);
    }
#undef RCG_CONV
    count_launch();
    RCG_CHECK_LAUNCH();
}

// Inference on B inputs [B][2][V] -> out [B][V], bfloat16 weights, in chunks
// of lanes so that the two ping-pong activation buffers stay small.
void Cnn::forward(cudaStream_t st, const float *in, int B, float *out, bool rounded) {
    const long long V = geom.V;
    const int chunk = (int)std::max<long long>(1, std::min<long long>(B, (64LL << 20) / (V * CMAX)));
    ensure(dact0, dact0_cap, (long long)chunk * CMAX * V);
    ensure(dact1, dact1_cap, (long long)chunk * CMAX * V);
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int nb = std::min(chunk, B - b0);
        const float *cur = in + (long long)b0 * CNN_CH[0] * V;
        for (int l = 0; l < CNN_LAYERS; ++l) {
            float *dst = l == CNN_LAYERS - 1 ? out + (long long)b0 * V : (l % 2 == 0 ? dact0 : dact1);
            conv(st, l, cur, dst, nb, l < CNN_LAYERS - 1, rounded);
            cur = dst;
        }
    }
}

// One training batch: forward with the master weights keeping every layer's
// output, mean squared error, backward into `grad`.  Returns nothing; the loss
// is accumulated into d_loss.
void Cnn::forward_backward(cudaStream_t st, const float *in, const float *tg, int B) {
    const long long V = geom.V;
    long long tot = 0;
    long long aoff[CNN_LAYERS + 1];
    aoff[0] = 0;
    for (int l = 0; l < CNN_LAYERS; ++l) aoff[l + 1] = aoff[l] + (long long)B * CNN_CH[l + 1] * V;
    tot = aoff[CNN_LAYERS];
    ensure(act, act_cap, tot);
    ensure(dact0, dact0_cap, (long long)B * CMAX * V);
    ensure(dact1, dact1_cap, (long long)B * CMAX * V);
    const float *cur = in;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        conv(st, l, cur, act + aoff[l], B, l < CNN_LAYERS - 1, false);
        cur = act + aoff[l];
    }
    // d(out) from the loss
    const float *outp = act + aoff[CNN_LAYERS - 1];
    k_mse<<<(int)std::min<long long>((B * V + 255) / 256, 1024), 256, 0, st>>>(outp, tg, dact0, (long long)B * V, d_loss);
    count_launch();
    RCG_CHECK_LAUNCH();
    float *g = dact0, *gnext = dact1;
    for (int l = CNN_LAYERS - 1; l >= 0; --l) {
        const int Cin = CNN_CH[l], Cout = CNN_CH[l + 1];
        const float *lin = l == 0 ? in : act + aoff[l - 1];
        k_conv3_bwd_w<<<Cout * Cin, 256, 0, st>>>(g, Cout, lin, Cin, grad + woff[l], grad + boff[l], B, geom.Gx,
                                                   geom.Gy, geom.Gz, V);
        count_launch();
        RCG_CHECK_LAUNCH();
        if (l > 0) {
            const size_t sm = sizeof(float) * (size_t)Cout * Cin * 27;
            dim3 grid((unsigned)((V + CT - 1) / CT), (unsigned)B);
            set_smem(k_conv3_bwd_data<16>, sm);
            k_conv3_bwd_data<16><<<grid, CT, sm, st>>>(g, Cout, theta + woff[l], act + aoff[l - 1], gnext, geom.Gx,
                                                         geom.Gy, geom.Gz, V);
            count_launch();
            RCG_CHECK_LAUNCH();
            std::swap(g, gnext);
        }
    }
}

double Cnn::gradient(cudaStream_t st, const float *in, const float *tg, int B) {
    RCG_CUDA_TRY(cudaMemsetAsync(d_loss, 0, sizeof(double), st));
    forward_backward(st, in, tg, B);
    double h = 0.0;
    RCG_CUDA_TRY(cudaMemcpyAsync(&h, d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    RCG_CUDA_TRY(cudaStreamSynchronize(st));
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
