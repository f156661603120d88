// The learned-augmentation U-Net on the 5th-generation tensor cores (not in
// the paper; the build's learned step, see cnn.cu for its place in the
// solve).  Three levels (the coarse grid, once and twice halved), 16-32-64
// channels, ten 3x3x3 zero-padded convolutions:
//
//   a0 = R(conv0(in))   s0 = R(conv1(a0))                      level 0, 16
//   a1 = R(conv2(down(s0)))   s1 = R(conv3(a1))               level 1, 32
//   a2 = R(conv4(down(s1)))                                    level 2, 64
//   a3 = R(conv5([up(a2), s1]))   a4 = R(conv6(a3))            level 1, 32
//   a5 = R(conv7([up(a4), s0]))   a6 = R(conv8(a5))            level 0, 16
//   out = conv9(a6)                                            level 0, 1
//
// R = ReLU, then rounding to bfloat16; down = mean over the cells of each
// 2x2x2 block inside the grid (dims ceil(G/2)), rounded to bfloat16; up =
// nearest-cell doubling, never materialised: the convolution reading an
// upsampled source addresses its parent cell.
//
// Activations are bfloat16, channels last ([batch][node][channel], 16, 32
// or 64 channels).  A convolution is an implicit GEMM on tcgen05.mma
// kind::f16 (bfloat16 operands, float32 accumulation in tensor memory):
//   M = 128 output nodes of one batch item per tile,
//   N = output channels (padded to a multiple of 16),
//   K = taps x input channels, in chunks of 64 channels (one 128-byte row
//       per node): 64 / C taps of a C-channel source per chunk.
// Per chunk every thread copies its node's 16-byte pieces (the source row at
// the tap's neighbour, zero-filled outside the grid) by cp.async straight
// into the 128-byte-swizzled K-major layout, beside the chunk's packed
// weights; one thread issues the four K = 16 MMAs and commits them to the
// stage's mbarrier; a ring of four stages, the copies two chunks ahead of the
// MMAs (so a stage is refilled two chunks after its MMAs were issued), three
// CTAs per SM at 16 output channels.  The epilogue reads the
// accumulator (tcgen05.ld), adds the bias, applies the ReLU or a ReLU mask
// (the backward pass) and stores bfloat16 or float32 channels-last rows.
//
// Training: the gradient with respect to a layer's input is the same kernel
// over the gradient of its output with the weights transposed and flipped
// (W'[ci][co][26 - d] = W[co][ci][d]); the weight gradient is a CUDA-core
// reduction over the nodes (k_unet_dw), float32 sums of bfloat16 operands.
// The bfloat16 roundings of the forward pass count as the identity in the
// backward pass, so the gradient approximates that of the exact network
// (float32 master weights) to bfloat16 precision.
//
// Every mbarrier wait is bounded: on timeout the CTA records
// RCG_ERR_TIMEOUT, waits (bounded) for the MMAs it issued, frees its tensor
// memory and returns.
#include "common.cuh"
#include "../../include/rcg.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

namespace rcg {

const int UNET_CIN[UNET_LAYERS] = {2, 16, 16, 32, 32, 96, 32, 48, 16, 16};
const int UNET_COUT[UNET_LAYERS] = {16, 16, 32, 32, 64, 32, 32, 16, 16, 1};

namespace {

using bf16 = __nv_bfloat16;

constexpr int UT = 128;                  // threads = tile rows (output nodes)
constexpr int UA_BYTES = UT * 128;       // A tile of one K-chunk: 128 rows x 64 bfloat16
constexpr int USTAGE = 4;
constexpr int UPF = 2;                   // chunks loaded ahead (the rest of the ring: MMAs in flight)
constexpr long long USPIN = 1LL << 22;   // polls of one mbarrier wait

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 16-byte piece c of row m in the 128-byte swizzle (8-row atoms of 1024 B)
__device__ __forceinline__ int swz(int m, int c) { return m * 128 + ((c ^ (m & 7)) << 4); }

// K-major tile in the 128-byte swizzle: 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: D float32, A and B bfloat16, both
// K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit_to(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool wait_bounded(uint32_t mbar, uint32_t parity, long long limit) {
    for (long long i = 0; i < limit; ++i)
        if (try_wait(mbar, parity)) return true;
    return false;
}

// 16 consecutive accumulator columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void cp16(void *dst, const void *src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst)), "l"(src), "r"(bytes) : "memory");
}

struct USrc {
    const bf16 *x;       // [B][Gz][Gy][Gx][C]
    int C;               // 16, 32 or 64
    int Gx, Gy, Gz;      // this source's grid
    int up;              // 1: read the parent cell (q >> 1) of output-grid node q
    int k0;              // first K-chunk of this source
};

struct UConv {
    USrc s[2];
    int nsrc, nchunk;
    const bf16 *Wp;      // packed weights [nchunk][NP][64]
    const float *bias;   // [Cout] or null
    int NP, Cout, relu;
    int Gx, Gy, Gz;      // output grid
    long long V;
    int B;
    bf16 *y;             // bfloat16 output [B][V][Cout] (Cout % 8 == 0), or null
    float *yf;           // float32 output [B][V][Cout], or null
    const bf16 *mask;    // y = acc * (mask > 0), [B][V][Cout], or null
    int *err;
};

__global__ void __launch_bounds__(UT, 1) k_unet_conv(UConv a) {
    extern __shared__ __align__(1024) char usm_raw[];
    __shared__ __align__(8) unsigned long long mbar[USTAGE];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_ok;
    char *smem = (char *)(((uintptr_t)usm_raw + 1023) & ~(uintptr_t)1023);
    const int stage_bytes = UA_BYTES + a.NP * 128;
    const uint32_t ncols = a.NP <= 32 ? 32u : a.NP <= 64 ? 64u : 128u;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < USTAGE; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_ok = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_bf16(UT, a.NP);
    const long long tiles_per = (a.V + UT - 1) / UT, ntiles = tiles_per * a.B;
    long long jj = 0;                 // chunks issued by this CTA before the current tile
    long long last = -1;              // global index of the last committed chunk (uniform)
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int b = (int)(tile / tiles_per);
        const long long p = (tile % tiles_per) * UT + threadIdx.x;    // this thread's output node
        const bool pin = p < a.V;
        int px = 0, py = 0, pz = 0;
        if (pin) {
            px = (int)(p % a.Gx);
            const long long t = p / a.Gx;
            py = (int)(t % a.Gy);
            pz = (int)(t / a.Gy);
        }
        // chunk k into the stage of global chunk index J
        auto load = [&](int k, long long J) {
            char *stg = smem + (int)(J % USTAGE) * stage_bytes;
            const int si = (a.nsrc > 1 && k >= a.s[1].k0) ? 1 : 0;
            const USrc &S = a.s[si];
            const int C = S.C, per = 64 / C, t0 = (k - S.k0) * per;
            const int pieces = C / 8;                  // 16-byte pieces per tap
#pragma unroll 1
            for (int u = 0; u < per; ++u) {
                const int tap = t0 + u;
                const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
                const int qx = px + dx, qy = py + dy, qz = pz + dz;
                const bool v = pin && tap < 27 && qx >= 0 && qx < a.Gx && qy >= 0 && qy < a.Gy && qz >= 0 &&
                               qz < a.Gz;
                const bf16 *src = S.x;
                if (v) {
                    const int sx = S.up ? qx >> 1 : qx, sy = S.up ? qy >> 1 : qy, sz = S.up ? qz >> 1 : qz;
                    src = S.x + ((((long long)b * S.Gz + sz) * S.Gy + sy) * S.Gx + sx) * C;
                }
                for (int c = 0; c < pieces; ++c)
                    cp16(stg + swz(threadIdx.x, u * pieces + c), v ? (const void *)(src + 8 * c) : (const void *)S.x,
                         v ? 16 : 0);
            }
            // the chunk's weights: NP rows of 128 bytes
            const bf16 *w = a.Wp + (long long)k * a.NP * 64;
            char *bt = stg + UA_BYTES;
            for (int e = threadIdx.x; e < a.NP * 8; e += UT) cp16(bt + swz(e >> 3, e & 7), w + 8 * e, 16);
        };
        for (int q = 0; q < UPF; ++q) {
            if (q < a.nchunk) load(q, jj + q);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        for (int k = 0; k < a.nchunk; ++k) {
            const long long J = jj + k;
            asm volatile("cp.async.wait_group %0;" ::"n"(UPF - 1) : "memory");      // chunk k landed (own copies)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();                                                        // ... everyone's
            if (!s_ok) { ok = false; break; }
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sa = su32(smem + (int)(J % USTAGE) * stage_bytes), sb = sa + UA_BYTES;
#pragma unroll
                for (int s = 0; s < 4; ++s)          // K = 16 per MMA = 32 bytes along the swizzled row
                    mma_bf16(tmem, desc_sw128(sa + 32 * s), desc_sw128(sb + 32 * s), idesc, (k > 0 || s > 0) ? 1u : 0u);
                commit_to(su32(&mbar[J % USTAGE]));
            }
            last = J;
            // chunk k + UPF refills the stage of chunk k + UPF - USTAGE, whose
            // MMAs were issued USTAGE - UPF iterations ago
            const int kw = k + UPF - USTAGE;
            if (kw >= 0) {
                const long long Jw = jj + kw;
                if (!wait_bounded(su32(&mbar[Jw % USTAGE]), (uint32_t)((Jw / USTAGE) & 1), USPIN)) {
                    s_ok = 0;
                    ok = false;
                }
            }
            if (ok && k + UPF < a.nchunk) load(k + UPF, J + UPF);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        // every thread takes the same branch from here (the epilogue's
        // tensor-memory loads are warp-collective)
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (!s_ok) ok = false;
        if (!ok) break;
        // the chunks not yet waited for (the last USTAGE - UPF): their MMAs
        // complete in issue order, the last one last
        for (int kw = std::max(0, a.nchunk - (USTAGE - UPF)); kw < a.nchunk; ++kw) {
            const long long Jw = jj + kw;
            if (!wait_bounded(su32(&mbar[Jw % USTAGE]), (uint32_t)((Jw / USTAGE) & 1), USPIN)) s_ok = 0;
        }
        last = -1;                                 // waited for with the full bound
        __syncthreads();
        if (!s_ok) { ok = false; break; }
        jj += a.nchunk;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // epilogue: row p of the accumulator is lane 32 warp + lane
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        const long long row = (long long)b * a.V + p;
        for (int c0 = 0; c0 < a.NP; c0 += 16) {
            float v[16];
            tmem_ld16(tl + (uint32_t)c0, v);
            if (!pin) continue;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int co = c0 + q;
                float t = v[q] + ((a.bias && co < a.Cout) ? a.bias[co] : 0.f);
                if (a.relu) t = fmaxf(t, 0.f);
                v[q] = t;
            }
            if (a.mask) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (c0 + 8 * h >= a.Cout) break;
                    const uint4 mk = *(const uint4 *)(a.mask + row * a.Cout + c0 + 8 * h);
                    const bf16 *m8 = (const bf16 *)&mk;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (!(__bfloat162float(m8[q]) > 0.f)) v[8 * h + q] = 0.f;
                }
            }
            if (a.y) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (c0 + 8 * h >= a.Cout) break;
                    uint4 o;
                    bf16 *o8 = (bf16 *)&o;
#pragma unroll
                    for (int q = 0; q < 8; ++q) o8[q] = __float2bfloat16_rn(v[8 * h + q]);
                    *(uint4 *)(a.y + row * a.Cout + c0 + 8 * h) = o;
                }
            }
            if (a.yf) {
                for (int q = 0; q < 16 && c0 + q < a.Cout; ++q) a.yf[row * a.Cout + c0 + q] = v[q];
            }
        }
        // the next tile's first MMA overwrites the accumulator: every thread's loads are done
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    // after a timeout: the last committed chunk (MMAs complete in issue order) before the memory is freed
    if (last >= 0) wait_bounded(su32(&mbar[last % USTAGE]), (uint32_t)((last / USTAGE) & 1), USPIN);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!ok) s_ok = 0;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (threadIdx.x == 0 && !s_ok) atomicExch(a.err, RCG_ERR_TIMEOUT);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// Packed weights of a convolution for the kernel above: Wp[k][n][kk] with
// chunk k of source s (channels C, first input channel ci0 of the layer,
// `creal` of them real, the rest zero padding) holding taps t0 .. t0 + 64/C - 1.
// Forward (flip = 0): Wp = W[n][ci0 + ci][tap] (n < Cout).  Transposed
// (flip = 1; the gradient with respect to the input, the source being the
// output gradient with C >= Cout channels): Wp[k][n][kk] = W[co][n][26 - tap]
// with co = kk mod C < Cout and n < Cin.  Values are rounded to bfloat16.
struct UPack {
    int k0, nk, C, ci0, creal;
};
__global__ void k_unet_pack(const float *__restrict__ W, int Cin, int Cout, UPack s0, UPack s1, int nsrc, int NP,
                            int flip, bf16 *__restrict__ Wp) {
    const int k = blockIdx.x;
    const UPack &S = (nsrc > 1 && k >= s1.k0) ? s1 : s0;
    const int per = 64 / S.C, t0 = (k - S.k0) * per;
    for (int e = threadIdx.x; e < NP * 64; e += blockDim.x) {
        const int n = e / 64, kk = e % 64;
        const int tap = t0 + kk / S.C, ci = kk % S.C;
        float v = 0.f;
        if (tap < 27 && ci < S.creal) {
            if (!flip) {
                if (n < Cout) v = W[((long long)n * Cin + S.ci0 + ci) * 27 + tap];
            } else if (n < Cin) {
                v = W[((long long)ci * Cin + n) * 27 + (26 - tap)];
            }
        }
        Wp[(long long)k * NP * 64 + e] = __float2bfloat16_rn(v);
    }
}

// [B][2][V] float32 features -> [B][V][16] bfloat16 (channels 2..15 zero)
__global__ void k_unet_input(const float *__restrict__ in, long long V, int B, bf16 *__restrict__ x) {
    const long long tot = (long long)B * V;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / V, v = e % V;
        uint4 o0 = make_uint4(0, 0, 0, 0), o1 = make_uint4(0, 0, 0, 0);
        bf16 *h = (bf16 *)&o0;
        h[0] = __float2bfloat16_rn(in[(b * 2) * V + v]);
        h[1] = __float2bfloat16_rn(in[(b * 2 + 1) * V + v]);
        *(uint4 *)(x + e * 16) = o0;
        *(uint4 *)(x + e * 16 + 8) = o1;
    }
}

// [B][V] float32 -> [B][V][16] bfloat16 in channel 0 (the output gradient of the last layer)
__global__ void k_unet_grad_out(const float *__restrict__ g, long long tot, bf16 *__restrict__ x) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        uint4 o0 = make_uint4(0, 0, 0, 0), o1 = make_uint4(0, 0, 0, 0);
        ((bf16 *)&o0)[0] = __float2bfloat16_rn(g[e]);
        *(uint4 *)(x + e * 16) = o0;
        *(uint4 *)(x + e * 16 + 8) = o1;
    }
}

// Level halving: y[b][k][c] = bf16(mean of x over the cells of block k inside the grid)
__global__ void k_unet_down(const bf16 *__restrict__ x, int C, int Gx, int Gy, int Gz, int B, bf16 *__restrict__ y) {
    const int Hx = (Gx + 1) / 2, Hy = (Gy + 1) / 2, Hz = (Gz + 1) / 2;
    const long long tot = (long long)B * Hz * Hy * Hx * C;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long t = e / C;
        const int kx = (int)(t % Hx); t /= Hx;
        const int ky = (int)(t % Hy); t /= Hy;
        const int kz = (int)(t % Hz);
        const long long b = t / Hz;
        float s = 0.f;
        int cnt = 0;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int z = 2 * kz + dz, y2 = 2 * ky + dy, x2 = 2 * kx + dx;
                    if (z < Gz && y2 < Gy && x2 < Gx) {
                        s += __bfloat162float(x[(((b * Gz + z) * Gy + y2) * Gx + x2) * C + c]);
                        ++cnt;
                    }
                }
        y[e] = __float2bfloat16_rn(s / (float)cnt);
    }
}

// Gradient of a level's activation a (C channels, grid G, B items), masked
// by a's ReLU: g = bf16((a > 0) * (direct + up^T(fine) + down^T(coarse)))
//   direct  d[b][v][doff + c] (float32, dC channels per row), same grid
//   up^T    sum over the (up to 8) cells of the doubled grid F whose parent
//           is v: f[b][child][foff + c] (fC channels per row)
//   down^T  h[b][parent(v)][hoff + c] / (cells of that parent inside G)
struct UGradTerm {
    const float *p;
    int Cs, off;
    int Fx, Fy, Fz;      // up^T: the fine grid
};
__global__ void k_unet_grad_mix(const bf16 *__restrict__ a, int C, int Gx, int Gy, int Gz, int B, UGradTerm direct,
                                UGradTerm upT, UGradTerm downT, bf16 *__restrict__ g) {
    const long long V = (long long)Gx * Gy * Gz, tot = (long long)B * V * C;
    const int Hx = (Gx + 1) / 2, Hy = (Gy + 1) / 2, Hz = (Gz + 1) / 2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const long long bv = e / C, b = bv / V, v = bv % V;
        const int x = (int)(v % Gx), y = (int)((v / Gx) % Gy), z = (int)(v / ((long long)Gx * Gy));
        float s = 0.f;
        if (direct.p) s += direct.p[bv * direct.Cs + direct.off + c];
        if (upT.p) {
            for (int dz = 0; dz < 2; ++dz)
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                        const int fz = 2 * z + dz, fy = 2 * y + dy, fx = 2 * x + dx;
                        if (fz < upT.Fz && fy < upT.Fy && fx < upT.Fx)
                            s += upT.p[(((b * upT.Fz + fz) * upT.Fy + fy) * upT.Fx + fx) * upT.Cs + upT.off + c];
                    }
        }
        if (downT.p) {
            const int kx = x >> 1, ky = y >> 1, kz = z >> 1;
            const int cnt = (min(2 * kx + 2, Gx) - 2 * kx) * (min(2 * ky + 2, Gy) - 2 * ky) * (min(2 * kz + 2, Gz) - 2 * kz);
            s += downT.p[(((b * Hz + kz) * Hy + ky) * Hx + kx) * downT.Cs + downT.off + c] / (float)cnt;
        }
        g[e] = __float2bfloat16_rn(__bfloat162float(a[e]) > 0.f ? s : 0.f);
    }
}

// Weight gradient of one source of a convolution at one tap (blockIdx.y):
// dW[co][ci0 + ci][tap] += sum over this CTA's nodes of
// g[b][p][co] x[b][p + tap][ci], for co < Cout, ci < creal.  g has Cg
// channels (>= Cout, zero padded), the source C.  Per block of DW_NODES
// nodes: the nodes' source rows (the tap's neighbour, or none outside the
// grid) are resolved once, both operands are staged in shared memory as
// float32 by 16-byte loads, then each thread accumulates a 4 x 4 block of
// (co, ci) over its share of the nodes.  The shares are summed in shared
// memory and added to dW once per CTA.
constexpr int DW_NODES = 128;
constexpr int DW_SMEM = 2 * DW_NODES * 64 * 4;
__global__ void __launch_bounds__(256)
k_unet_dw(const bf16 *__restrict__ g, int Cg, int Cout, const bf16 *__restrict__ x, int C, int creal, int ci0, int Cin,
          int Sx, int Sy, int Sz, int up, int Gx, int Gy, int Gz, int B, long long per_cta, float *__restrict__ dW) {
    extern __shared__ float4 dw_sm4[];
    float *gs = (float *)dw_sm4;                      // [DW_NODES][Cg]
    float *xs = gs + DW_NODES * 64;                   // [DW_NODES][C]
    __shared__ long long s_src[DW_NODES];             // row of x for the node (-1: zero), row of g
    __shared__ long long s_row[DW_NODES];
    const int tap = blockIdx.y;
    const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
    const int V = Gx * Gy * Gz;
    const long long tot = (long long)B * V;
    const long long e0 = (long long)blockIdx.x * per_cta, e1 = min(e0 + per_cta, tot);
    const int nbc = Cg / 4, nbi = C / 4, nblk = nbc * nbi;         // 4 x 4 blocks
    const int groups = max(1, 256 / nblk);
    const int blk = threadIdx.x % nblk, grp = threadIdx.x / nblk;
    const bool act = threadIdx.x < groups * nblk;
    const int bc = (blk / nbi) * 4, bi = (blk % nbi) * 4;
    const int pg = Cg / 8, px8 = C / 8;                            // 16-byte pieces per row
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.f;
    for (long long n0 = e0; n0 < e1; n0 += DW_NODES) {
        if (threadIdx.x < DW_NODES) {
            const long long e = n0 + threadIdx.x;
            long long src = -1, row = -1;
            if (e < e1) {
                row = e;
                const int b = (int)(e / V), v = (int)(e - (long long)b * V);
                const int px = v % Gx, t = v / Gx, py = t % Gy, pz = t / Gy;
                const int qx = px + dx, qy = py + dy, qz = pz + dz;
                if (qx >= 0 && qx < Gx && qy >= 0 && qy < Gy && qz >= 0 && qz < Gz) {
                    const int sx = up ? qx >> 1 : qx, sy = up ? qy >> 1 : qy, sz = up ? qz >> 1 : qz;
                    src = (((long long)b * Sz + sz) * Sy + sy) * Sx + sx;
                }
            }
            s_src[threadIdx.x] = src;
            s_row[threadIdx.x] = row;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < DW_NODES * (pg + px8); t += 256) {
            const int node = t % DW_NODES, part = t / DW_NODES;
            float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float *dst;
            if (part < pg) {
                const long long row = s_row[node];
                if (row >= 0) {
                    const uint4 q = *(const uint4 *)(g + row * Cg + 8 * part);
                    const bf16 *h = (const bf16 *)&q;
#pragma unroll
                    for (int i = 0; i < 8; ++i) f[i] = __bfloat162float(h[i]);
                }
                dst = gs + node * Cg + 8 * part;
            } else {
                const int pc = part - pg;
                const long long src = s_src[node];
                if (src >= 0) {
                    const uint4 q = *(const uint4 *)(x + src * C + 8 * pc);
                    const bf16 *h = (const bf16 *)&q;
#pragma unroll
                    for (int i = 0; i < 8; ++i) f[i] = __bfloat162float(h[i]);
                }
                dst = xs + node * C + 8 * pc;
            }
            *(float4 *)dst = make_float4(f[0], f[1], f[2], f[3]);
            *(float4 *)(dst + 4) = make_float4(f[4], f[5], f[6], f[7]);
        }
        __syncthreads();
        if (act) {
            for (int node = grp; node < DW_NODES; node += groups) {
                const float4 gv = *(const float4 *)(gs + node * Cg + bc);
                const float4 xv = *(const float4 *)(xs + node * C + bi);
                const float ga[4] = {gv.x, gv.y, gv.z, gv.w}, xa[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i * 4 + j] += ga[i] * xa[j];
            }
        }
        __syncthreads();
    }
    // sum the node groups' shares in shared memory (gs is free now), then one
    // atomic per (co, ci) and CTA
    float *red = gs;                                  // [16][nblk]
    for (int t = threadIdx.x; t < 16 * nblk; t += 256) red[t] = 0.f;
    __syncthreads();
    if (act) {
#pragma unroll
        for (int i = 0; i < 16; ++i) atomicAdd(&red[i * nblk + blk], acc[i]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 16 * nblk; t += 256) {
        const int i = t / nblk, k = t % nblk;
        const int co = (k / nbi) * 4 + i / 4, ci = (k % nbi) * 4 + i % 4;
        if (co < Cout && ci < creal) atomicAdd(&dW[((long long)co * Cin + ci0 + ci) * 27 + tap], red[t]);
    }
}

// db[co] += sum over nodes of g[b][p][co] (co < Cout of Cg channels)
__global__ void __launch_bounds__(256) k_unet_db(const bf16 *__restrict__ g, int Cg, int Cout, long long tot,
                                                 float *__restrict__ db) {
    __shared__ float s[64];
    if (threadIdx.x < 64) s[threadIdx.x] = 0.f;
    __syncthreads();
    const int c = threadIdx.x % Cg, rows = 256 / Cg;
    float acc = 0.f;
    for (long long e = (long long)blockIdx.x * rows + threadIdx.x / Cg; e < tot; e += (long long)gridDim.x * rows)
        acc += __bfloat162float(g[e * Cg + c]);
    if (threadIdx.x < rows * Cg) atomicAdd(&s[c], acc);
    __syncthreads();
    if (threadIdx.x < Cout) atomicAdd(&db[threadIdx.x], s[threadIdx.x]);
}

int grid_for(long long work, int per = 256) {
    return (int)std::max<long long>(1, std::min<long long>((work + per - 1) / per, 152LL * 16));
}

}  // namespace

// ------------------------------------------------------------------ host side
UNet::UNet(int Gx_, int Gy_, int Gz_) {
    G[0][0] = Gx_; G[0][1] = Gy_; G[0][2] = Gz_;
    for (int l = 1; l < 3; ++l)
        for (int a = 0; a < 3; ++a) G[l][a] = (G[l - 1][a] + 1) / 2;
    for (int l = 0; l < 3; ++l) V[l] = (long long)G[l][0] * G[l][1] * G[l][2];
    int o = 0;
    for (int l = 0; l < UNET_LAYERS; ++l) {
        woff[l] = o;
        o += UNET_COUT[l] * UNET_CIN[l] * 27;
        boff[l] = o;
        o += UNET_COUT[l];
    }
    P = o;
    // sources of each layer: (buffer, level, channels, up) and the packed layout
    static const int lvl_out[UNET_LAYERS] = {0, 0, 1, 1, 2, 1, 1, 0, 0, 0};
    for (int l = 0; l < UNET_LAYERS; ++l) {
        Layer &L = lay[l];
        L.lvl = lvl_out[l];
        L.Cout = UNET_COUT[l];
        L.NP = (L.Cout + 15) / 16 * 16;
        L.Cin = UNET_CIN[l];
        L.NPb = (L.Cin + 15) / 16 * 16;
    }
    // (channels of each source, padded to 16 / 32 / 64; concatenations: up first)
    auto src = [&](int l, int i, int C, int creal, int up) {
        lay[l].sC[i] = C; lay[l].sreal[i] = creal; lay[l].sup[i] = up;
    };
    src(0, 0, 16, 2, 0); lay[0].nsrc = 1;
    src(1, 0, 16, 16, 0); lay[1].nsrc = 1;
    src(2, 0, 16, 16, 0); lay[2].nsrc = 1;
    src(3, 0, 32, 32, 0); lay[3].nsrc = 1;
    src(4, 0, 32, 32, 0); lay[4].nsrc = 1;
    src(5, 0, 64, 64, 1); src(5, 1, 32, 32, 0); lay[5].nsrc = 2;
    src(6, 0, 32, 32, 0); lay[6].nsrc = 1;
    src(7, 0, 32, 32, 1); src(7, 1, 16, 16, 0); lay[7].nsrc = 2;
    src(8, 0, 16, 16, 0); lay[8].nsrc = 1;
    src(9, 0, 16, 16, 0); lay[9].nsrc = 1;
    long long fo = 0, bo = 0;
    for (int l = 0; l < UNET_LAYERS; ++l) {
        Layer &L = lay[l];
        int k = 0, ci0 = 0;
        for (int i = 0; i < L.nsrc; ++i) {
            L.sk0[i] = k;
            L.sci0[i] = ci0;
            k += (27 + 64 / L.sC[i] - 1) / (64 / L.sC[i]);
            ci0 += L.sreal[i];
        }
        L.nchunk = k;
        L.pack_f = fo;
        fo += (long long)L.nchunk * L.NP * 64;
        // transposed: one source, the output gradient with Cg = NP channels (>= 16)
        L.Cg = L.NP;
        L.nchunk_b = (27 + 64 / L.Cg - 1) / (64 / L.Cg);
        L.pack_b = bo;
        bo += (long long)L.nchunk_b * L.NPb * 64;
    }
    RCG_CUDA_TRY(cudaMalloc(&wpf, sizeof(bf16) * (size_t)fo));
    RCG_CUDA_TRY(cudaMalloc(&wpb, sizeof(bf16) * (size_t)bo));
    RCG_CUDA_TRY(cudaMalloc(&d_err, sizeof(int)));
    RCG_CUDA_TRY(cudaMemset(d_err, 0, sizeof(int)));
}

UNet::~UNet() {
    for (void *p : std::vector<void *>{wpf, wpb, d_err, abuf, gbuf, fbuf})
        if (p) cudaFree(p);
}

void UNet::grow(void *&p, long long &cap, long long bytes) {
    if (bytes <= cap) return;
    if (p) RCG_CUDA_TRY(cudaFree(p));
    p = nullptr;
    cap = 0;
    RCG_CUDA_TRY(cudaMalloc(&p, (size_t)bytes));
    cap = bytes;
}

void UNet::pack(cudaStream_t st, const float *theta, bool backward) {
    for (int l = 0; l < UNET_LAYERS; ++l) {
        const Layer &L = lay[l];
        UPack s0{L.sk0[0], 0, L.sC[0], L.sci0[0], L.sreal[0]};
        UPack s1{L.sk0[1], 0, L.sC[1], L.sci0[1], L.sreal[1]};
        k_unet_pack<<<L.nchunk, 256, 0, st>>>(theta + woff[l], L.Cin, L.Cout, s0, s1, L.nsrc, L.NP, 0,
                                               (bf16 *)wpf + L.pack_f);
        count_launch();
        RCG_CHECK_LAUNCH();
        if (backward && l > 0) {
            UPack sb{0, 0, L.Cg, 0, L.Cout};
            k_unet_pack<<<L.nchunk_b, 256, 0, st>>>(theta + woff[l], L.Cin, L.Cout, sb, sb, 1, L.NPb, 1,
                                                     (bf16 *)wpb + L.pack_b);
            count_launch();
            RCG_CHECK_LAUNCH();
        }
    }
}

// activation buffers of B items: offsets (elements of bfloat16) per tensor
void UNet::layout(int B) {
    long long o = 0;
    auto put = [&](int id, int lvl, int C) {
        aoff[id] = o;
        o += (long long)B * V[lvl] * C;
        o = (o + 63) / 64 * 64;
    };
    put(A_IN, 0, 16);
    put(A_A0, 0, 16);
    put(A_S0, 0, 16);
    put(A_P0, 1, 16);
    put(A_A1, 1, 32);
    put(A_S1, 1, 32);
    put(A_P1, 2, 32);
    put(A_A2, 2, 64);
    put(A_A3, 1, 32);
    put(A_A4, 1, 32);
    put(A_A5, 0, 16);
    put(A_A6, 0, 16);
    grow(abuf, abuf_cap, o * (long long)sizeof(bf16));
}

void UNet::conv(cudaStream_t st, int l, const bf16 *s0, const bf16 *s1, const float *bias, bool relu, bf16 *y,
                float *yf, const bf16 *mask, int B, bool backward, const bf16 *wp_override) {
    const Layer &L = lay[l];
    UConv a{};
    const int lo = L.lvl;
    a.Gx = G[lo][0]; a.Gy = G[lo][1]; a.Gz = G[lo][2];
    a.V = V[lo];
    a.B = B;
    if (!backward) {
        static const int lvl_in[UNET_LAYERS][2] = {{0, 0}, {0, 0}, {1, 0}, {1, 0}, {2, 0}, {2, 1}, {1, 0}, {1, 0},
                                                   {0, 0}, {0, 0}};
        for (int i = 0; i < L.nsrc; ++i) {
            const int li = lvl_in[l][i];
            a.s[i] = USrc{i == 0 ? s0 : s1, L.sC[i], G[li][0], G[li][1], G[li][2], L.sup[i], L.sk0[i]};
        }
        a.nsrc = L.nsrc;
        a.nchunk = L.nchunk;
        a.Wp = (const bf16 *)wpf + L.pack_f;
        a.NP = L.NP;
        a.Cout = L.Cout;
    } else {
        // the gradient with respect to the layer's (stacked) input, on the output grid
        a.s[0] = USrc{s0, L.Cg, G[lo][0], G[lo][1], G[lo][2], 0, 0};
        a.nsrc = 1;
        a.nchunk = L.nchunk_b;
        a.Wp = wp_override ? wp_override : (const bf16 *)wpb + L.pack_b;
        a.NP = L.NPb;
        a.Cout = L.Cin == 2 ? 16 : L.Cin;
    }
    a.bias = bias;
    a.relu = relu ? 1 : 0;
    a.y = y;
    a.yf = yf;
    a.mask = mask;
    a.err = d_err;
    const int smem = USTAGE * (UA_BYTES + a.NP * 128) + 1024;
    static bool attr_done[64] = {};
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {   // function attributes hold per device
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_unet_conv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          USTAGE * (UA_BYTES + 128 * 128) + 1024));
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_unet_conv, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    // resident CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per
    // CTA) and tensor memory (512 columns per SM)
    const int ncols = a.NP <= 32 ? 32 : a.NP <= 64 ? 64 : 128;
    const int occ = std::max(1, std::min({(228 * 1024) / (smem + 2048), 512 / ncols, 4}));
    const long long tiles = (a.V + UT - 1) / UT * B;
    const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, 152LL * occ));
    k_unet_conv<<<grid, UT, smem, st>>>(a);
    count_launch();
    RCG_CHECK_LAUNCH();
}

const bf16 *UNet::act(int id) const { return (const bf16 *)abuf + aoff[id]; }
bf16 *UNet::actw(int id) { return (bf16 *)abuf + aoff[id]; }

void UNet::down(cudaStream_t st, const bf16 *x, int C, int lvl, int B, bf16 *y) {
    const long long work = (long long)B * V[lvl + 1] * C;
    k_unet_down<<<grid_for(work), 256, 0, st>>>(x, C, G[lvl][0], G[lvl][1], G[lvl][2], B, y);
    count_launch();
    RCG_CHECK_LAUNCH();
}

// forward over B items in[B][2][V0] (float32) -> out[B][V0] (float32); the
// activations stay in abuf (for the backward pass)
void UNet::forward(cudaStream_t st, const float *theta, const float *in, int B, float *out) {
    layout(B);
    k_unet_input<<<grid_for((long long)B * V[0]), 256, 0, st>>>(in, V[0], B, actw(A_IN));
    count_launch();
    RCG_CHECK_LAUNCH();
    const float *bia[UNET_LAYERS];
    for (int l = 0; l < UNET_LAYERS; ++l) bia[l] = theta + boff[l];
    conv(st, 0, act(A_IN), nullptr, bia[0], true, actw(A_A0), nullptr, nullptr, B);
    conv(st, 1, act(A_A0), nullptr, bia[1], true, actw(A_S0), nullptr, nullptr, B);
    down(st, act(A_S0), 16, 0, B, actw(A_P0));
    conv(st, 2, act(A_P0), nullptr, bia[2], true, actw(A_A1), nullptr, nullptr, B);
    conv(st, 3, act(A_A1), nullptr, bia[3], true, actw(A_S1), nullptr, nullptr, B);
    down(st, act(A_S1), 32, 1, B, actw(A_P1));
    conv(st, 4, act(A_P1), nullptr, bia[4], true, actw(A_A2), nullptr, nullptr, B);
    conv(st, 5, act(A_A2), act(A_S1), bia[5], true, actw(A_A3), nullptr, nullptr, B);
    conv(st, 6, act(A_A3), nullptr, bia[6], true, actw(A_A4), nullptr, nullptr, B);
    conv(st, 7, act(A_A4), act(A_S0), bia[7], true, actw(A_A5), nullptr, nullptr, B);
    conv(st, 8, act(A_A5), nullptr, bia[8], true, actw(A_A6), nullptr, nullptr, B);
    conv(st, 9, act(A_A6), nullptr, bia[9], false, nullptr, out, nullptr, B);
}

// Gradient of the loss with respect to the master weights (grad, zeroed
// here) from dout[B][V0] = d loss / d out, after forward() on the same batch.
void UNet::backward(cudaStream_t st, const float *dout, int B, float *grad) {
    RCG_CUDA_TRY(cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)P, st));
    const long long V0 = V[0], V1 = V[1], V2 = V[2];
    // bfloat16 gradient buffers (16-64 channels) and one float32 buffer for
    // the stacked-input gradients
    const long long gb = (long long)B * std::max({V0 * 16, V1 * 64, V2 * 64});
    grow(gbuf, gbuf_cap, 3 * gb * (long long)sizeof(bf16));
    // float32 input gradients: f_a layer 7's [up(a4), s0] (48 channels, level
    // 0), f_b layer 5's [up(a2), s1] (96, level 1) and later layer 2's (16,
    // level 1), f_c layer 4's (32, level 2)
    const long long fa = (long long)B * V0 * 48, fb = (long long)B * V1 * 96, fc = (long long)B * V2 * 32;
    grow(fbuf, fbuf_cap, (fa + fb + fc) * (long long)sizeof(float));
    bf16 *g_a = (bf16 *)gbuf, *g_b = g_a + gb, *g_c = g_b + gb;
    float *f_a = (float *)fbuf, *f_b = f_a + fa, *f_c = f_b + fb;
    auto dw = [&](int l, const bf16 *g, int i, const bf16 *x) {
        const Layer &L = lay[l];
        static const int lvl_in[UNET_LAYERS][2] = {{0, 0}, {0, 0}, {1, 0}, {1, 0}, {2, 0}, {2, 1}, {1, 0}, {1, 0},
                                                   {0, 0}, {0, 0}};
        const int lo = L.lvl, li = lvl_in[l][i];
        const long long tot = (long long)B * V[lo];
        // node chunks of at least 16 blocks: ~5-8 CTAs per SM over the 27 taps
        const long long per = std::max<long long>(DW_NODES * 16, (tot + 47) / 48 / DW_NODES * DW_NODES);
        dim3 gr((unsigned)((tot + per - 1) / per), 27);
        static bool attr[64] = {};
        int dev = 0;
        RCG_CUDA_TRY(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64 || !attr[dev]) {
            RCG_CUDA_TRY(cudaFuncSetAttribute(k_unet_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, DW_SMEM));
            if (dev >= 0 && dev < 64) attr[dev] = true;
        }
        k_unet_dw<<<gr, 256, DW_SMEM, st>>>(g, L.Cg, L.Cout, x, L.sC[i], L.sreal[i], L.sci0[i], L.Cin, G[li][0],
                                             G[li][1], G[li][2], L.sup[i], G[lo][0], G[lo][1], G[lo][2], B, per,
                                             grad + woff[l]);
        count_launch();
        RCG_CHECK_LAUNCH();
        if (i == 0) {
            k_unet_db<<<grid_for(tot, 16), 256, 0, st>>>(g, L.Cg, L.Cout, tot, grad + boff[l]);
            count_launch();
            RCG_CHECK_LAUNCH();
        }
    };
    auto mix = [&](const bf16 *a, int C, int lvl, UGradTerm d, UGradTerm u, UGradTerm h, bf16 *g) {
        const long long work = (long long)B * V[lvl] * C;
        k_unet_grad_mix<<<grid_for(work), 256, 0, st>>>(a, C, G[lvl][0], G[lvl][1], G[lvl][2], B, d, u, h, g);
        count_launch();
        RCG_CHECK_LAUNCH();
    };
    const UGradTerm none{nullptr, 0, 0, 0, 0, 0};
    // layer 9 (no ReLU): g9 = dout in channel 0 of 16
    k_unet_grad_out<<<grid_for((long long)B * V0), 256, 0, st>>>(dout, (long long)B * V0, g_a);
    count_launch();
    RCG_CHECK_LAUNCH();
    dw(9, g_a, 0, act(A_A6));
    conv(st, 9, g_a, nullptr, nullptr, false, g_b, nullptr, act(A_A6), B, true);      // g8
    dw(8, g_b, 0, act(A_A5));
    conv(st, 8, g_b, nullptr, nullptr, false, g_c, nullptr, act(A_A5), B, true);      // g7
    dw(7, g_c, 0, act(A_A4));
    dw(7, g_c, 1, act(A_S0));
    conv(st, 7, g_c, nullptr, nullptr, false, nullptr, f_a, nullptr, B, true);        // d[up(a4), s0], 48 ch
    mix(act(A_A4), 32, 1, none, UGradTerm{f_a, 48, 0, G[0][0], G[0][1], G[0][2]}, none, g_a);   // g6
    dw(6, g_a, 0, act(A_A3));
    conv(st, 6, g_a, nullptr, nullptr, false, g_b, nullptr, act(A_A3), B, true);      // g5
    dw(5, g_b, 0, act(A_A2));
    dw(5, g_b, 1, act(A_S1));
    conv(st, 5, g_b, nullptr, nullptr, false, nullptr, f_b, nullptr, B, true);        // d[up(a2), s1], 96 ch
    mix(act(A_A2), 64, 2, none, UGradTerm{f_b, 96, 0, G[1][0], G[1][1], G[1][2]}, none, g_a);   // g4
    dw(4, g_a, 0, act(A_P1));
    conv(st, 4, g_a, nullptr, nullptr, false, nullptr, f_c, nullptr, B, true);
    mix(act(A_S1), 32, 1, UGradTerm{f_b, 96, 64, 0, 0, 0}, none, UGradTerm{f_c, 32, 0, 0, 0, 0}, g_c);   // g3
    dw(3, g_c, 0, act(A_A1));
    conv(st, 3, g_c, nullptr, nullptr, false, g_b, nullptr, act(A_A1), B, true);      // g2
    dw(2, g_b, 0, act(A_P0));
    conv(st, 2, g_b, nullptr, nullptr, false, nullptr, f_b, nullptr, B, true);        // d(down(s0)), 16 ch, level 1
    mix(act(A_S0), 16, 0, UGradTerm{f_a, 48, 32, 0, 0, 0}, none, UGradTerm{f_b, 16, 0, 0, 0, 0}, g_a);   // g1
    dw(1, g_a, 0, act(A_A0));
    conv(st, 1, g_a, nullptr, nullptr, false, g_b, nullptr, act(A_A0), B, true);      // g0
    dw(0, g_b, 0, act(A_IN));
}

int UNet::error(cudaStream_t st) {
    int h = 0;
    RCG_CUDA_TRY(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RCG_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) RCG_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    return h;
}

}  // namespace rcg
