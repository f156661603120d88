// Tall-skinny products C (+)= A^T B on the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulators in tensor memory), for the basis
// products of the ordered append (Sec. 5.3 incremental QR: V^T W, W^T W,
// V^T Q, Q^T Q with n-long columns) and the seed's Gram matrices.
//
// A (n x ka) and B (n x kb) are float32, column-major (each column
// contiguous along n: K-major operands for the MMA).  A CTA owns a 128 x 128
// output tile and a slice of n (split-K), walked in K-steps of 32 rows:
//
//   * cp.async copies the raw 128 x 32 tiles of A and B straight into the
//     128-byte-swizzled K-major layout (row m = one column of A: 32 floats =
//     128 B; 16-byte chunk c of row m stored at chunk c ^ (m mod 8)), two
//     K-steps ahead, into a 3-stage ring;
//   * every value x is split in place into hi = rn_tf32(x) and, beside it,
//     lo = rn_tf32(x - hi); three MMAs per 8-deep K-slice (hi hi, hi lo,
//     lo hi) give products at float32 level ("3xTF32");
//   * one thread issues the 12 MMAs of a K-step into one of two tensor-memory
//     accumulators and commits them to an mbarrier;
//   * while the tensor core runs step k, the CTA drains step k-1's
//     accumulator into registers.  Each step's accumulator starts from zero,
//     so the tensor core never adds a small product into a large sum (its
//     float32 accumulation is not round-to-nearest: a long accumulation of
//     same-sign products drifts by ~1 ulp per MMA); the registers sum the
//     per-step partials in two levels (16 steps, then the slice).
//
// The float32 tile of every slice goes to a scratch [z][kb][ka]; a second
// kernel sums the slices in float64 into C.  Symmetric products (A == B)
// compute the upper tiles only and mirror them.
//
// Every mbarrier wait is bounded: on timeout the CTA records RCG_ERR_TIMEOUT
// in *err, stops issuing work, waits (bounded) for its MMAs and copies,
// frees its tensor memory and returns.
#include "common.cuh"
#include "../../include/rcg.h"

#include <algorithm>
#include <cstdint>
#include <mutex>

namespace rcg {
namespace {

constexpr int TM = 128;                 // output rows per CTA (columns of A)
constexpr int TNc = 128;                // output columns per CTA (columns of B)
constexpr int TBK = 32;                 // K rows per step (one 128-byte swizzle row)
constexpr int NTHR = 256;               // 8 warps
constexpr int TILE_BYTES = TM * TBK * 4;                 // 16 KiB
constexpr int STAGE_BYTES = 4 * TILE_BYTES;              // A hi, B hi, A lo, B lo
constexpr int NSTAGE = 3;
constexpr int WBYTES = TBK * 8;                          // the step's float64 row weights
constexpr int TC_SMEM = NSTAGE * STAGE_BYTES + NSTAGE * WBYTES + 1024;   // + 1024-byte alignment slack
constexpr int LEVEL1 = 16;              // K-steps summed before the second level
constexpr long long SPIN_LIMIT = 1LL << 22;

// Polls of a main-loop mbarrier wait: the calling context's
// rcg_options.spin_budget when positive, SPIN_LIMIT when 0, none when
// negative (every main-loop wait runs out at once).  The final wait for the
// last committed step always has the full SPIN_LIMIT.
long long spin_budget() { return g_spin_budget > 0 ? g_spin_budget : g_spin_budget < 0 ? 0 : SPIN_LIMIT; }
constexpr long long LIST_MIN_CHUNK = 8;  // fewest K-steps per slice when a block list sets the length
constexpr int NUM_SMS = 152;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle
// layout: 8-row groups 1024 B apart (stride byte offset), descriptor
// version 1 (tcgen05), layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused by swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: D f32, A and B tf32, both K-major, M x N.
__host__ __device__ constexpr uint32_t make_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
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

// bounded wait (at most `limit` polls); returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

// Round a float32 to the nearest TF32 value (10 explicit mantissa bits),
// ties away from zero, on the bit pattern: add half of the dropped range to
// the magnitude bits and clear them (finite inputs; two integer operations,
// where the conversion instruction would run on a slower pipe).
__device__ __forceinline__ float rn_tf32(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// 16-byte chunk c (K rows 4c..4c+3) of tile row m, 128-byte swizzle.
__device__ __forceinline__ int sw_off(int m, int c) { return m * 128 + ((c ^ (m & 7)) << 4); }

// Copy the raw 128 x 32 tile of X at rows k0..k0+31 into `dst` (zero-filled
// outside the matrix and past row k1).  Thread t copies 16-byte chunk t%8 of
// columns c0 + t/8 + 32 it (it = 0..3); `colp` = X + (c0 + t/8) ldx + 4 (t%8),
// `ncol` = number of those four columns inside the matrix.
__device__ __forceinline__ void prefetch_tile(const float *colp, long long step_col, int ncol, long long k0,
                                              long long k1, char *dst) {
    const int m0 = threadIdx.x >> 3, c = threadIdx.x & 7;
    const long long k = k0 + 4 * c;
    const long long left = k1 - k;
    const int bytes_row = left >= 4 ? 16 : (left > 0 ? (int)(4 * left) : 0);
#pragma unroll
    for (int it = 0; it < TM * (TBK / 4) / NTHR; ++it) {
        const int bytes = it < ncol ? bytes_row : 0;
        const float *src = bytes ? colp + it * step_col + k0 : colp;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst + sw_off(m0 + 32 * it, c))),
                     "l"(src), "r"(bytes)
                     : "memory");
    }
}

// The step's 32 row weights (float64) into `dst` (zero past row n).
__device__ __forceinline__ void prefetch_w(const double *wt, long long k0, long long n, char *dst) {
    if (threadIdx.x < WBYTES / 16) {
        const long long k = k0 + 2 * threadIdx.x;
        const int bytes = k + 2 <= n ? 16 : (k < n ? 8 : 0);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst + 16 * threadIdx.x)),
                     "l"(bytes ? wt + k : wt), "r"(bytes)
                     : "memory");
    }
}

// hi in place, lo at the same offset in `lo`; with row weights w (the step's
// 32 float64 weights in shared memory) every value is first scaled by its
// row's weight.  16-byte chunk o of the tile holds rows 4 c .. 4 c + 3 with
// c = ((o / 16) mod 8) xor (m mod 8), m = o / 128 (the 128-byte swizzle).
// WEIGHTED is a template argument so that the unweighted split carries no
// weight arithmetic at all (not even predicated off); the scale multiplies in
// float32 ((float)w * 1.0f == (float)w exactly).
template <bool WEIGHTED>
__device__ __forceinline__ void split_tile(char *hi, char *lo, const double *w = nullptr, float wscale = 1.f) {
#pragma unroll
    for (int it = 0; it < TILE_BYTES / 16 / NTHR; ++it) {
        const int o = (threadIdx.x + it * NTHR) * 16;
        float4 v = *(const float4 *)(hi + o);
        if constexpr (WEIGHTED) {
            const int m = o >> 7, c = ((o >> 4) & 7) ^ (m & 7);
            v.x *= (float)w[4 * c] * wscale; v.y *= (float)w[4 * c + 1] * wscale;
            v.z *= (float)w[4 * c + 2] * wscale; v.w *= (float)w[4 * c + 3] * wscale;
        }
        float4 h, l;
        h.x = rn_tf32(v.x); h.y = rn_tf32(v.y); h.z = rn_tf32(v.z); h.w = rn_tf32(v.w);
        l.x = rn_tf32(v.x - h.x); l.y = rn_tf32(v.y - h.y); l.z = rn_tf32(v.z - h.z); l.w = rn_tf32(v.w - h.w);
        *(float4 *)(hi + o) = h;
        *(float4 *)(lo + o) = l;
    }
}

// 32 consecutive accumulator columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// K-steps per slice when the weights' block list (nsteps blocks) is spread
// over z slices; slices past the last block hold no partial.
__device__ __forceinline__ long long list_chunk(long long nsteps, int z) {
    const long long c = (nsteps + z - 1) / z;
    return c < LIST_MIN_CHUNK ? LIST_MIN_CHUNK : c;
}

__global__ void __launch_bounds__(NTHR, 1)
k_tc_tn(long long n, const float *__restrict__ A, long long lda, int ka, const float *__restrict__ B, long long ldb,
        int kb, int symmetric, float *__restrict__ part, long long chunk, int *__restrict__ err,
        const double *__restrict__ wt, const int *__restrict__ blist, const int *__restrict__ bcount, int zper,
        long long ldw_b, long long ldl_b, double wscale, long long spin) {
    if (symmetric && blockIdx.x > blockIdx.y) return;        // lower tiles are mirrored by the reduction
    extern __shared__ __align__(1024) char smem_raw[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_ok;
    char *smem = (char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    char *wsm = smem + NSTAGE * STAGE_BYTES;
    const int i0 = blockIdx.x * TM, j0 = blockIdx.y * TNc;
    // K-steps of this slice: steps s_begin .. s_begin + nk - 1 (chunk = steps per
    // slice); step s covers rows 32 s .. 32 s + 31, or rows 32 blist[s] .. with a
    // block list (the blocks where the weights do not vanish)
    // batch bk = blockIdx.z / zper (weights wt + bk ldw_b, block list
    // blist + bk ldl_b with count bcount[bk]), slice bz = blockIdx.z mod zper
    const int bk = blockIdx.z / zper, bz = blockIdx.z % zper;
    if (wt) wt += bk * ldw_b;
    if (blist) { blist += bk * ldl_b; bcount += bk; }
    const long long nsteps = blist ? (long long)*bcount : (n + TBK - 1) / TBK;
    if (blist) {                       // the support, not n, sets the slice length
        chunk = list_chunk(nsteps, zper);
        if ((long long)bz * chunk >= nsteps) return;            // empty slice: the reduction skips it
    }
    const long long s_begin = (long long)bz * chunk;
    const long long s_end = s_begin + chunk < nsteps ? s_begin + chunk : nsteps;
    const long long nk = s_end > s_begin ? s_end - s_begin : 0;
    auto step_row = [&](long long ks) -> long long {
        return (long long)TBK * (blist ? (long long)blist[s_begin + ks] : s_begin + ks);
    };
    auto step_end = [&](long long k0) -> long long { return k0 + TBK < n ? k0 + TBK : n; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(2 * TNc));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_ok = 1;
    }
    // this thread's source columns (see prefetch_tile)
    const int mt = threadIdx.x >> 3;
    const float *colA = A + (long long)(i0 + mt < ka ? i0 + mt : 0) * lda + 4 * (threadIdx.x & 7);
    const float *colB = B + (long long)(j0 + mt < kb ? j0 + mt : 0) * ldb + 4 * (threadIdx.x & 7);
    const int ncolA = i0 + mt < ka ? min(4, (ka - i0 - mt + 31) / 32) : 0;
    const int ncolB = j0 + mt < kb ? min(4, (kb - j0 - mt + 31) / 32) : 0;
    const long long stepA = 32 * lda, stepB = 32 * ldb;
    // prologue: steps 0 and 1 in flight (one cp.async group per step; empty
    // groups keep the count uniform)
    for (int q = 0; q < 2; ++q) {
        if (q < nk) {
            char *stg = smem + q * STAGE_BYTES;
            const long long k0 = step_row(q);
            prefetch_tile(colA, stepA, ncolA, k0, step_end(k0), stg);
            prefetch_tile(colB, stepB, ncolB, k0, step_end(k0), stg + TILE_BYTES);
            if (wt) prefetch_w(wt, k0, n, wsm + q * WBYTES);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = make_idesc_tf32(TM, TNc);
    // accumulator lane block of this warp and this thread's 64 columns
    const uint32_t t_lane = (uint32_t)((warp & 3) * 32) << 16;
    const int col0 = (warp >> 2) * 64;
    float acc1[64], acc2[64];
#pragma unroll
    for (int q = 0; q < 64; ++q) { acc1[q] = 0.f; acc2[q] = 0.f; }
    bool ok = true;
    long long drained = 0;                // steps whose partial is in acc1 / acc2
    long long last = -1;                  // last step whose MMAs were committed (the same in every thread)
    auto drain = [&](long long q) {       // the MMAs of step q are complete
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t base = tmem + t_lane + (uint32_t)((q & 1) * TNc + col0);
        float v[32];
        tmem_ld32(base, v);
#pragma unroll
        for (int c = 0; c < 32; ++c) acc1[c] += v[c];
        tmem_ld32(base + 32, v);
#pragma unroll
        for (int c = 0; c < 32; ++c) acc1[32 + c] += v[c];
        if (((q + 1) % LEVEL1) == 0) {
#pragma unroll
            for (int c = 0; c < 64; ++c) { acc2[c] += acc1[c]; acc1[c] = 0.f; }
        }
        drained = q + 1;
    };
    for (long long ks = 0; ks < nk; ++ks) {
        char *stg = smem + (int)(ks % NSTAGE) * STAGE_BYTES;
        asm volatile("cp.async.wait_group 1;" ::: "memory");      // step ks has landed (own copies)
        __syncthreads();                                           // ... everyone's; s_ok is uniform here
        if (!s_ok) { ok = false; break; }
        if (wt)                                                    // A hi | A lo (weighted rows)
            split_tile<true>(stg, stg + 2 * TILE_BYTES, (const double *)(wsm + (int)(ks % NSTAGE) * WBYTES),
                             (float)wscale);
        else
            split_tile<false>(stg, stg + 2 * TILE_BYTES);
        split_tile<false>(stg + TILE_BYTES, stg + 3 * TILE_BYTES); // B hi | B lo
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t d = tmem + (uint32_t)((ks & 1) * TNc);
            const uint32_t a_hi = smem_u32(stg), b_hi = a_hi + TILE_BYTES;
            const uint32_t a_lo = a_hi + 2 * TILE_BYTES, b_lo = a_hi + 3 * TILE_BYTES;
#pragma unroll
            for (int s = 0; s < TBK / 8; ++s) {        // K = 8 per MMA = 32 bytes along the swizzled row
                const uint32_t o = s * 32;
                mma_tf32(d, make_desc_sw128(a_hi + o), make_desc_sw128(b_hi + o), idesc, s > 0 ? 1u : 0u);
                mma_tf32(d, make_desc_sw128(a_hi + o), make_desc_sw128(b_lo + o), idesc, 1u);
                mma_tf32(d, make_desc_sw128(a_lo + o), make_desc_sw128(b_hi + o), idesc, 1u);
            }
            mma_commit(smem_u32(&mbar[ks & 1]));
        }
        last = ks;
        // step ks-1: its MMAs free the stage that step ks+2 is copied into, and
        // its accumulator is drained while step ks runs on the tensor core
        if (ks >= 1) {
            const long long q = ks - 1;
            if (mbar_wait(smem_u32(&mbar[q & 1]), (uint32_t)((q >> 1) & 1), spin)) {
                drain(q);
            } else {
                s_ok = 0;
                ok = false;
            }
        }
        if (ok && ks + 2 < nk) {
            char *nxt = smem + (int)((ks + 2) % NSTAGE) * STAGE_BYTES;
            const long long k0 = step_row(ks + 2);
            prefetch_tile(colA, stepA, ncolA, k0, step_end(k0), nxt);
            prefetch_tile(colB, stepB, ncolB, k0, step_end(k0), nxt + TILE_BYTES);
            if (wt) prefetch_w(wt, k0, n, wsm + (int)((ks + 2) % NSTAGE) * WBYTES);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    // the last committed step: wait for its MMAs with the full bound, also
    // after a main-loop timeout (the MMAs complete in issue order, so none
    // runs on the tensor memory when it is freed); every earlier step was
    // waited for in the loop, so the barrier's phase parity is unambiguous
    if (last >= 0) {
        const bool done = mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1), SPIN_LIMIT);
        if (ok && done && last == nk - 1 && drained == nk - 1) drain(last);
        else ok = false;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");          // no copy in flight at exit
    if (!ok) s_ok = 0;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (threadIdx.x == 0 && !s_ok) atomicExch(err, RCG_ERR_TIMEOUT);
    // this thread's row of the slice: row i0 + (warp&3)*32 + lane, 64 columns
    float *dst = part + (long long)blockIdx.z * ((long long)kb * ka);
    const int row = i0 + (warp & 3) * 32 + lane;
    if (s_ok && row < ka) {
#pragma unroll
        for (int c = 0; c < 64; ++c) {
            const int col = j0 + col0 + c;
            if (col < kb) dst[(long long)col * ka + row] = acc2[c] + acc1[c];
        }
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TNc));
}

// Ascending list of the 32-row blocks where w does not vanish, in two
// passes.  k_block_flags: one warp per (vector, block) writes 1 / 0 into the
// list slot of the block (one coalesced 256-byte read per block).
__global__ void k_block_flags(long long n, const double *__restrict__ w, int *__restrict__ list, int nvec,
                              long long ldw, long long ldl) {
    const long long nb = (n + TBK - 1) / TBK;
    const long long total = nb * nvec;
    const int lane = threadIdx.x & 31;
    for (long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw < total;
         gw += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long v = gw / nb, b = gw % nb;
        const long long k = b * TBK + lane;
        const bool nz = k < n && w[v * ldw + k] != 0.0;
        const unsigned any = __ballot_sync(0xffffffffu, nz);
        if (lane == 0) list[v * ldl + b] = any != 0u;
    }
}

// k_block_compact: CTA v compacts the flags of vector v in place, in chunks
// of 1024 x 8 flags: every flag of a chunk is in registers before any index
// of it is written, and an index never lands past its own flag's slot.
__global__ void __launch_bounds__(1024) k_block_compact(long long n, int *__restrict__ list, int *__restrict__ count,
                                                        long long ldl) {
    constexpr int PER = 8;
    __shared__ int scan[1024];
    list += blockIdx.x * ldl;
    const long long nb = (n + TBK - 1) / TBK;
    int base = 0;
    for (long long c0 = 0; c0 < nb; c0 += 1024 * PER) {
        const long long b0 = c0 + (long long)threadIdx.x * PER;
        int f[PER], cnt = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            f[i] = b0 + i < nb ? list[b0 + i] : 0;
            cnt += f[i];
        }
        scan[threadIdx.x] = cnt;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {       // inclusive scan
            const int v = threadIdx.x >= (unsigned)o ? scan[threadIdx.x - o] : 0;
            __syncthreads();
            scan[threadIdx.x] += v;
            __syncthreads();
        }
        int pos = base + scan[threadIdx.x] - cnt;
#pragma unroll
        for (int i = 0; i < PER; ++i)
            if (f[i]) list[pos++] = (int)(b0 + i);
        base += scan[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) count[blockIdx.x] = base;
}

// ------------------------------------------------------------------ NN
// Out (n x m, float32) = alpha V C + beta Out with V (n x k, float32,
// column-major) and C (k x m, float64): the basis updates of the append
// (W -= V (V^T W), Q = W R^-1, V <- Q R2^-1).  A CTA owns 128 rows x 128
// columns of Out and walks k in steps of 32.  C is split once per call into
// TF32 hi / lo rows (k_nn_prep_b, rows of ldb floats) that cp.async copies
// straight into the swizzled K-major B operand; the V tile arrives in its
// natural row-major-in-n layout and is transposed into the K-major A operand
// while it is split.  Accumulation and drains as in k_tc_tn.
constexpr int NN_RAW = TBK * TM * 4;                                   // raw V tile: [32 k][128 rows]
constexpr int NN_SMEM = NSTAGE * STAGE_BYTES + 2 * NN_RAW + 1024;

__global__ void k_nn_prep_b(const double *__restrict__ C, int ldc, int k, int m, float *__restrict__ Bh,
                            float *__restrict__ Bl, int ldb) {
    const long long tot = (long long)m * ldb;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / ldb), kk = (int)(e % ldb);
        const float b = kk < k ? (float)C[kk + (long long)j * ldc] : 0.f;
        const float h = rn_tf32(b);
        Bh[e] = h;
        Bl[e] = rn_tf32(b - h);
    }
}

__global__ void __launch_bounds__(NTHR, 1)
k_tc_nn(long long n, const float *__restrict__ V, long long ldv, int k, const float *__restrict__ Bh,
        const float *__restrict__ Bl, int ldb, int m, float *__restrict__ Out, long long ldo, float alpha, float beta,
        int *__restrict__ err, long long spin) {
    extern __shared__ __align__(1024) char smem_raw[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_ok;
    char *smem = (char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    char *rawA = smem + NSTAGE * STAGE_BYTES;
    const long long i0 = (long long)blockIdx.x * TM;
    const int j0 = blockIdx.y * TNc;
    const long long nk = (k + TBK - 1) / TBK;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(2 * TNc));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_ok = 1;
    }
    // this thread's B rows (columns j0 + t/8 + 32 it of Out) in the prepared hi / lo arrays
    const int mt = threadIdx.x >> 3;
    const long long stepB = 32LL * ldb;
    const float *colBh = Bh + (long long)(j0 + mt < m ? j0 + mt : 0) * ldb + 4 * (threadIdx.x & 7);
    const float *colBl = Bl + (long long)(j0 + mt < m ? j0 + mt : 0) * ldb + 4 * (threadIdx.x & 7);
    const int ncolB = j0 + mt < m ? min(4, (m - j0 - mt + 31) / 32) : 0;
    auto prefetch = [&](long long q) {
        const long long k0 = q * TBK;
        // V tile: [kk][128 rows], 32 16-byte chunks per k column
        char *ra = rawA + (int)(q & 1) * NN_RAW;
#pragma unroll
        for (int it = 0; it < (TBK * TM / 4) / NTHR; ++it) {
            const int e = threadIdx.x + it * NTHR;
            const int kk = e >> 5, c = e & 31;
            const long long row = i0 + 4 * c, col = k0 + kk;
            int bytes = 0;
            const float *src = V;
            if (col < k && row < n) {
                src = V + col * ldv + row;
                bytes = n - row >= 4 ? 16 : (int)(4 * (n - row));
            }
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(ra + kk * 512 + c * 16)),
                         "l"(src), "r"(bytes)
                         : "memory");
        }
        // B hi / lo rows straight into the operand stage (128-byte swizzle)
        char *stg = smem + (int)(q % NSTAGE) * STAGE_BYTES;
        prefetch_tile(colBh, stepB, ncolB, k0, (long long)ldb, stg + TILE_BYTES);
        prefetch_tile(colBl, stepB, ncolB, k0, (long long)ldb, stg + 3 * TILE_BYTES);
    };
    for (int q = 0; q < 2; ++q) {
        if (q < nk) prefetch(q);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = make_idesc_tf32(TM, TNc);
    const uint32_t t_lane = (uint32_t)((warp & 3) * 32) << 16;
    const int col0 = (warp >> 2) * 64;
    float acc1[64], acc2[64];
#pragma unroll
    for (int q = 0; q < 64; ++q) { acc1[q] = 0.f; acc2[q] = 0.f; }
    bool ok = true;
    long long drained = 0;
    long long last = -1;                  // last step whose MMAs were committed (the same in every thread)
    auto drain = [&](long long q) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t base = tmem + t_lane + (uint32_t)((q & 1) * TNc + col0);
        float v[32];
        tmem_ld32(base, v);
#pragma unroll
        for (int c = 0; c < 32; ++c) acc1[c] += v[c];
        tmem_ld32(base + 32, v);
#pragma unroll
        for (int c = 0; c < 32; ++c) acc1[32 + c] += v[c];
        if (((q + 1) % LEVEL1) == 0) {
#pragma unroll
            for (int c = 0; c < 64; ++c) { acc2[c] += acc1[c]; acc1[c] = 0.f; }
        }
        drained = q + 1;
    };
    for (long long ks = 0; ks < nk; ++ks) {
        char *stg = smem + (int)(ks % NSTAGE) * STAGE_BYTES;
        const char *ra = rawA + (int)(ks & 1) * NN_RAW;
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        if (!s_ok) { ok = false; break; }
        // split and transpose: thread (t, row) takes k = 4t..4t+3 of one row
#pragma unroll
        for (int it = 0; it < (TBK / 4) * TM / NTHR; ++it) {
            const int e = threadIdx.x + it * NTHR;
            const int row = e & 127, t = e >> 7;
            float4 h, l;
            float x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = *(const float *)(ra + (4 * t + q) * 512 + row * 4);
            h.x = rn_tf32(x[0]); h.y = rn_tf32(x[1]); h.z = rn_tf32(x[2]); h.w = rn_tf32(x[3]);
            l.x = rn_tf32(x[0] - h.x); l.y = rn_tf32(x[1] - h.y); l.z = rn_tf32(x[2] - h.z); l.w = rn_tf32(x[3] - h.w);
            *(float4 *)(stg + sw_off(row, t)) = h;
            *(float4 *)(stg + 2 * TILE_BYTES + sw_off(row, t)) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t d = tmem + (uint32_t)((ks & 1) * TNc);
            const uint32_t a_hi = smem_u32(stg), b_hi = a_hi + TILE_BYTES;
            const uint32_t a_lo = a_hi + 2 * TILE_BYTES, b_lo = a_hi + 3 * TILE_BYTES;
#pragma unroll
            for (int s = 0; s < TBK / 8; ++s) {
                const uint32_t o = s * 32;
                mma_tf32(d, make_desc_sw128(a_hi + o), make_desc_sw128(b_hi + o), idesc, s > 0 ? 1u : 0u);
                mma_tf32(d, make_desc_sw128(a_hi + o), make_desc_sw128(b_lo + o), idesc, 1u);
                mma_tf32(d, make_desc_sw128(a_lo + o), make_desc_sw128(b_hi + o), idesc, 1u);
            }
            mma_commit(smem_u32(&mbar[ks & 1]));
        }
        last = ks;
        if (ks >= 1) {
            const long long q = ks - 1;
            if (mbar_wait(smem_u32(&mbar[q & 1]), (uint32_t)((q >> 1) & 1), spin)) {
                drain(q);
            } else {
                s_ok = 0;
                ok = false;
            }
        }
        // step ks+2: the raw V stage of step ks (split above) and the operand
        // stage of step ks-1 (its MMAs are complete) are free
        if (ok && ks + 2 < nk) prefetch(ks + 2);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    if (last >= 0) {                      // as in k_tc_tn: the last committed step, full bound
        const bool done = mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1), SPIN_LIMIT);
        if (ok && done && last == nk - 1 && drained == nk - 1) drain(last);
        else ok = false;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!ok) s_ok = 0;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (threadIdx.x == 0 && !s_ok) atomicExch(err, RCG_ERR_TIMEOUT);
    const long long row = i0 + (warp & 3) * 32 + lane;
    if (s_ok && row < n) {
        // all loads of Out before the first store: a store between them would
        // serialise one DRAM latency per column (the columns may alias for
        // all the compiler knows)
        const int ncol = min(64, m - j0 - col0);
        float *o = Out + (long long)(j0 + col0) * ldo + row;
#pragma unroll
        for (int c = 0; c < 64; ++c) acc2[c] = alpha * (acc2[c] + acc1[c]);
        if (beta != 0.f) {
#pragma unroll
            for (int c = 0; c < 64; ++c) acc1[c] = c < ncol ? o[(long long)c * ldo] : 0.f;
#pragma unroll
            for (int c = 0; c < 64; ++c) acc2[c] += beta * acc1[c];
        }
#pragma unroll
        for (int c = 0; c < 64; ++c)
            if (c < ncol) o[(long long)c * ldo] = acc2[c];
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TNc));
}

// C[i + j*ldc] (+)= sum_z part[z][j][i] in float64; a symmetric product
// reads the lower tiles from the mirrored upper ones.
// Batch bk of nbatch: C + bk ldcb from the partials part + bk zper tot.
__global__ void k_tc_reduce(const float *__restrict__ part, int zper, int ka, int kb, int symmetric,
                            double *__restrict__ C, int ldc, int accumulate, const int *__restrict__ bcount,
                            int nbatch, long long ldcb) {
    const long long tot = (long long)ka * kb;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot * nbatch;
         e += (long long)gridDim.x * blockDim.x) {
        const int bk = (int)(e / tot);
        const long long el = e % tot;
        int z = zper;
        if (bcount) {                  // only the slices that held blocks of the list
            const long long nsteps = bcount[bk];
            const long long chunk = list_chunk(nsteps, zper);
            z = (int)((nsteps + chunk - 1) / chunk);
        }
        const int i = (int)(el % ka), j = (int)(el / ka);
        const long long src = (symmetric && i / TM > j / TNc) ? (long long)i * ka + j : el;
        const float *pb = part + (long long)bk * zper * tot;
        double s = 0.0;
        for (int q = 0; q < z; ++q) s += (double)pb[(long long)q * tot + src];
        double *c = C + bk * ldcb + i + (long long)j * ldc;
        *c = accumulate ? *c + s : s;
    }
}

}  // namespace

// Slices z of the long dimension for (n, ka, kb) and the float scratch they
// need: one CTA per SM, z chosen so that the CTAs fill whole waves.
long long tc_gemm_tn_scratch(long long n, int ka, int kb, bool symmetric, int *z_out, long long *chunk_out) {
    const long long tx = (ka + TM - 1) / TM, ty = (kb + TNc - 1) / TNc;
    const long long tiles = symmetric ? tx * (tx + 1) / 2 : tx * ty;
    long long z = 1;
    if (n > 0) {
        const long long zmax = std::max<long long>(1, n / 512);    // at least 512 rows per slice
        double best = -1.0;
        for (long long zz = 1; zz <= std::min<long long>(zmax, 4 * NUM_SMS); ++zz) {
            const long long ctas = tiles * zz;
            const long long waves = (ctas + NUM_SMS - 1) / NUM_SMS;
            const double eff = (double)ctas / (double)(waves * NUM_SMS);
            if (eff > best + 0.02) { best = eff; z = zz; }
            if (waves > 3) break;
        }
    }
    const long long steps = (n + TBK - 1) / TBK;
    long long chunk = steps > 0 ? (steps + z - 1) / z : 1;      // K-steps per slice
    if (steps > 0) z = (steps + chunk - 1) / chunk;
    if (z_out) *z_out = (int)z;
    if (chunk_out) *chunk_out = chunk;
    return z * (long long)ka * kb;
}

// Blocks of 32 rows where w is not zero (list: (n + 31) / 32 ints; count: 1 int).
void tc_block_list(cudaStream_t st, long long n, const double *w, int *list, int *count, int nvec, long long ldw,
                   long long ldl) {
    if (nvec <= 0) return;
    const long long warps = ((n + TBK - 1) / TBK) * nvec;
    k_block_flags<<<(unsigned)std::min<long long>((warps * 32 + 255) / 256, 8 * NUM_SMS), 256, 0, st>>>(
        n, w, list, nvec, ldw, ldl ? ldl : (n + TBK - 1) / TBK);
    count_launch();
    RCG_CHECK_LAUNCH();
    k_block_compact<<<nvec, 1024, 0, st>>>(n, list, count, ldl ? ldl : (n + TBK - 1) / TBK);
    count_launch();
    RCG_CHECK_LAUNCH();
}

// The copies need 16-byte aligned columns.
bool tc_gemm_tn_ok(long long lda, long long ldb, const void *A, const void *B) {
    return lda % 4 == 0 && ldb % 4 == 0 && ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0;
}

// C (ka x kb, ld ldc) = / += A^T B with A, B float32 column-major (n rows,
// 16-byte aligned, lda and ldb multiples of 4).  symmetric: A == B, ka == kb.
// scratch: >= tc_gemm_tn_scratch(...) floats; err: device int (0 = ok).
void tc_gemm_tn(cudaStream_t st, long long n, const float *A, long long lda, int ka, const float *B, long long ldb,
                int kb, double *C, int ldc, bool accumulate, bool symmetric, float *scratch, int *err,
                const double *wt, const int *blist, const int *bcount) {
    if (ka <= 0 || kb <= 0) return;
    if (!tc_gemm_tn_ok(lda, ldb, A, B)) throw Error{RCG_ERR_INVALID, "tc_gemm_tn: operands not 16-byte aligned"};
    if (symmetric && (A != B || ka != kb || lda != ldb)) throw Error{RCG_ERR_INVALID, "tc_gemm_tn: not symmetric"};
    int z;
    long long chunk;
    tc_gemm_tn_scratch(n, ka, kb, symmetric, &z, &chunk);
    static bool attr[64] = {};          // per device ordinal
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_tc_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    dim3 grid((ka + TM - 1) / TM, (kb + TNc - 1) / TNc, z);
    if ((blist != nullptr) != (bcount != nullptr) || (blist && !wt)) throw Error{RCG_ERR_INVALID, "tc_gemm_tn: block list"};
    k_tc_tn<<<grid, NTHR, TC_SMEM, st>>>(n, A, lda, ka, B, ldb, kb, symmetric ? 1 : 0, scratch, chunk, err, wt, blist,
                                         bcount, z, 0, 0, 1.0, spin_budget());
    count_launch();
    RCG_CHECK_LAUNCH();
    const long long tot = (long long)ka * kb;
    const int blocks = (int)std::min<long long>((tot + 255) / 256, 2048);
    k_tc_reduce<<<blocks, 256, 0, st>>>(scratch, z, ka, kb, symmetric ? 1 : 0, C, ldc, accumulate ? 1 : 0, bcount, 1,
                                        0);
    count_launch();
    RCG_CHECK_LAUNCH();
}

// Slices per batch and float scratch of tc_gram_w_batched.
long long tc_gram_w_batched_scratch(int ka, int nbatch, int *zper_out) {
    const long long tx = (ka + TM - 1) / TM;
    const long long tiles = tx * (tx + 1) / 2;
    long long zper = (4LL * NUM_SMS + tiles * nbatch - 1) / (tiles * nbatch);
    if (zper < 1) zper = 1;
    if (zper_out) *zper_out = (int)zper;
    return zper * nbatch * (long long)ka * ka;
}

// C_b (+)= A^T diag(wscale w_b) A (ka x ka, ld ldc, C_b = C + b ldcb) for
// b < nbatch in one launch: w_b = wt + b ldw with block lists blist + b ldl,
// counts bcount[b] (tc_block_list); the slices of each batch follow its
// support.  The weights are copied 16 bytes at a time: wt 16-byte aligned,
// ldw even.
void tc_gram_w_batched(cudaStream_t st, long long n, const float *A, long long lda, int ka, double *C, int ldc,
                       long long ldcb, int nbatch, const double *wt, long long ldw, const int *blist, long long ldl,
                       const int *bcount, float *scratch, int *err, bool accumulate, double wscale) {
    if (ka <= 0 || nbatch <= 0) return;
    if (!tc_gemm_tn_ok(lda, lda, A, A) || !wt || !blist || !bcount || ((uintptr_t)wt & 15) || (ldw & 1))
        throw Error{RCG_ERR_INVALID, "tc_gram_w_batched: bad operands"};
    int zper;
    tc_gram_w_batched_scratch(ka, nbatch, &zper);
    static bool attr[64] = {};
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_tc_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    const unsigned tx = (unsigned)((ka + TM - 1) / TM);
    // grid z holds zper slices per batch and may not exceed 65535: chunks of batches
    const int bmax = std::max(1, 65535 / zper);
    for (int b0 = 0; b0 < nbatch; b0 += bmax) {
        const int nb = std::min(bmax, nbatch - b0);
        dim3 grid(tx, tx, (unsigned)(zper * nb));
        k_tc_tn<<<grid, NTHR, TC_SMEM, st>>>(n, A, lda, ka, A, lda, ka, 1, scratch, 1, err, wt + b0 * ldw,
                                             blist + b0 * ldl, bcount + b0, zper, ldw, ldl, wscale, spin_budget());
        count_launch();
        RCG_CHECK_LAUNCH();
        const long long tot = (long long)ka * ka * nb;
        const int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
        k_tc_reduce<<<blocks, 256, 0, st>>>(scratch, zper, ka, ka, 1, C + b0 * ldcb, ldc, accumulate ? 1 : 0,
                                            bcount + b0, nb, ldcb);
        count_launch();
        RCG_CHECK_LAUNCH();
    }
}

// Prepared-B float32 scratch of tc_gemm_nn: 2 m ldb floats, ldb = k rounded up to 32.
long long tc_gemm_nn_scratch(int k, int m) { return 2LL * m * ((k + TBK - 1) / TBK * TBK); }

// Out (n x m, ld ldo) = alpha V C + beta Out on the tensor cores (3xTF32).
// V: float32 n x k (ld ldv, 16-byte aligned columns); C: float64 k x m (ld ldc).
void tc_gemm_nn(cudaStream_t st, long long n, const float *V, long long ldv, int k, const double *C, int ldc, int m,
                float *Out, long long ldo, double alpha, double beta, float *scratch, int *err) {
    if (m <= 0 || n <= 0) return;
    if (k <= 0 || ldv % 4 != 0 || ((uintptr_t)V & 15)) throw Error{RCG_ERR_INVALID, "tc_gemm_nn: bad operands"};
    const int ldb = (k + TBK - 1) / TBK * TBK;
    float *Bh = scratch, *Bl = scratch + (long long)m * ldb;
    const long long tot = (long long)m * ldb;
    k_nn_prep_b<<<(unsigned)std::min<long long>((tot + 255) / 256, 2048), 256, 0, st>>>(C, ldc, k, m, Bh, Bl, ldb);
    count_launch();
    RCG_CHECK_LAUNCH();
    static bool attr[64] = {};
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_tc_nn, cudaFuncAttributeMaxDynamicSharedMemorySize, NN_SMEM));
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    dim3 grid((unsigned)((n + TM - 1) / TM), (unsigned)((m + TNc - 1) / TNc));
    k_tc_nn<<<grid, NTHR, NN_SMEM, st>>>(n, V, ldv, k, Bh, Bl, ldb, m, Out, ldo, (float)alpha, (float)beta, err,
                                         spin_budget());
    count_launch();
    RCG_CHECK_LAUNCH();
}

}  // namespace rcg

// ------------------------------------------------------------ C ABI
namespace {
// Split-K scratch and timeout flag of rcg_gemm_tn_f32, one per device, grown
// on demand and kept until exit; the mutex is held for the whole call (which
// waits for its stream), so concurrent host threads take turns.
std::mutex g_gemm_mu;
float *g_gemm_scr[64] = {};
long long g_gemm_cap[64] = {};
int *g_gemm_err[64] = {};
int *g_gemm_bl[64] = {};
long long g_gemm_blcap[64] = {};
}  // namespace

extern "C" int rcg_gemm_tn_f32(const float *A, long long lda, int ka, const float *B, long long ldb, int kb,
                               long long n, const double *w, double *C, int ldc, int engine, int symmetric,
                               void *stream) {
    using namespace rcg;
    if ((n > 0 && (!A || !B)) || !C || ka < 0 || kb < 0 || n < 0 || lda < n || ldb < n || ldc < ka ||
        (engine != 0 && engine != 1))
        return RCG_ERR_INVALID;
    if (symmetric && (A != B || ka != kb || lda != ldb)) return RCG_ERR_INVALID;
    if (engine == 1 && !tc_gemm_tn_ok(lda, ldb, A, B)) return RCG_ERR_INVALID;
    if (w && ((uintptr_t)w & 15)) return RCG_ERR_INVALID;
    if (ka == 0 || kb == 0) return RCG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_gemm_mu);
    int rc = RCG_OK;
    try {
        int dev = 0;
        RCG_CUDA_TRY(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64) return RCG_ERR_INVALID;
        if (engine == 1) {
            const long long need = tc_gemm_tn_scratch(n, ka, kb, symmetric != 0, nullptr, nullptr);
            if (need > g_gemm_cap[dev]) {
                if (g_gemm_scr[dev]) RCG_CUDA_TRY(cudaFree(g_gemm_scr[dev]));
                g_gemm_scr[dev] = nullptr;
                g_gemm_cap[dev] = 0;
                RCG_CUDA_TRY(cudaMalloc(&g_gemm_scr[dev], sizeof(float) * (size_t)need));
                g_gemm_cap[dev] = need;
            }
            if (!g_gemm_err[dev]) RCG_CUDA_TRY(cudaMalloc(&g_gemm_err[dev], sizeof(int)));
            RCG_CUDA_TRY(cudaMemsetAsync(g_gemm_err[dev], 0, sizeof(int), st));
            int *bl = nullptr;
            if (w) {
                const long long nb = (n + TBK - 1) / TBK;
                if (nb + 1 > g_gemm_blcap[dev]) {
                    if (g_gemm_bl[dev]) RCG_CUDA_TRY(cudaFree(g_gemm_bl[dev]));
                    g_gemm_bl[dev] = nullptr;
                    g_gemm_blcap[dev] = 0;
                    RCG_CUDA_TRY(cudaMalloc(&g_gemm_bl[dev], sizeof(int) * (size_t)(nb + 1)));
                    g_gemm_blcap[dev] = nb + 1;
                }
                bl = g_gemm_bl[dev];
                tc_block_list(st, n, w, bl + 1, bl);
            }
            tc_gemm_tn(st, n, A, lda, ka, B, ldb, kb, C, ldc, false, symmetric != 0, g_gemm_scr[dev], g_gemm_err[dev],
                       w, bl ? bl + 1 : nullptr, bl);
        } else if (w) {
            gemm_tn_acc<float, float, double>(st, n, A, lda, ka, B, ldb, kb, C, ldc, false, w);
        } else {
            gemm_tn<float, float>(st, n, A, lda, ka, B, ldb, kb, C, ldc, false);
        }
        RCG_CUDA_TRY(cudaStreamSynchronize(st));
        if (engine == 1) {
            int h = 0;
            RCG_CUDA_TRY(cudaMemcpy(&h, g_gemm_err[dev], sizeof(int), cudaMemcpyDeviceToHost));
            if (h) rc = RCG_ERR_TIMEOUT;
        }
    } catch (const Error &e) {
        rc = e.code;
    }
    return rc;
}

extern "C" int rcg_gemm_nn_f32(const float *V, long long ldv, int k, const double *C, int ldc, int m, long long n,
                               float *Out, long long ldo, double alpha, double beta, int engine, void *stream) {
    using namespace rcg;
    if ((n > 0 && k > 0 && (!V || !C)) || (n > 0 && m > 0 && !Out) || k < 0 || m < 0 || n < 0 || ldv < n || ldo < n ||
        ldc < k || (engine != 0 && engine != 1))
        return RCG_ERR_INVALID;
    if (engine == 1 && (ldv % 4 != 0 || ((uintptr_t)V & 15))) return RCG_ERR_INVALID;
    if (m == 0 || n == 0) return RCG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_gemm_mu);
    int rc = RCG_OK;
    try {
        int dev = 0;
        RCG_CUDA_TRY(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64) return RCG_ERR_INVALID;
        if (engine == 1 && k > 0) {
            const long long need = tc_gemm_nn_scratch(k, m);
            if (need > g_gemm_cap[dev]) {
                if (g_gemm_scr[dev]) RCG_CUDA_TRY(cudaFree(g_gemm_scr[dev]));
                g_gemm_scr[dev] = nullptr;
                g_gemm_cap[dev] = 0;
                RCG_CUDA_TRY(cudaMalloc(&g_gemm_scr[dev], sizeof(float) * (size_t)need));
                g_gemm_cap[dev] = need;
            }
            if (!g_gemm_err[dev]) RCG_CUDA_TRY(cudaMalloc(&g_gemm_err[dev], sizeof(int)));
            RCG_CUDA_TRY(cudaMemsetAsync(g_gemm_err[dev], 0, sizeof(int), st));
            tc_gemm_nn(st, n, V, ldv, k, C, ldc, m, Out, ldo, alpha, beta, g_gemm_scr[dev], g_gemm_err[dev]);
        } else {
            gemm_nn<float, float>(st, n, V, ldv, k, C, ldc, m, Out, ldo, alpha, beta);
        }
        RCG_CUDA_TRY(cudaStreamSynchronize(st));
        if (engine == 1 && k > 0) {
            int h = 0;
            RCG_CUDA_TRY(cudaMemcpy(&h, g_gemm_err[dev], sizeof(int), cudaMemcpyDeviceToHost));
            if (h) rc = RCG_ERR_TIMEOUT;
        }
    } catch (const Error &e) {
        rc = e.code;
    }
    return rc;
}
