// Float32 inner iteration of the batched deflated CG (see cg.cu for the
// recurrences) for grids with Nx % 4 == 0, restructured for HBM bandwidth:
//
//   k_stencil4   q = A~_s p, float4 along x, one active lane per CTA row,
//                fused p^T q
//   k_stencil4z  the same for 3D grids, two lanes per CTA, planes streamed
//                through a shared-memory ring (each value read about once)
//   k_update4    x += alpha p, r -= alpha q, fused r^T r and the private
//                (A W)^T r dots, float4; whole waves of CTAs over the
//                flattened (lane, node block) range
//   k_u0dots     (A~_s U_0)^T r (or U_0^T r at a restart) for a tile of
//                <= 32 lanes of one sample: a shared-memory tiled product,
//                so each A~_s U_0 element is read once per tile
//   k_mu         per lane (one warp): convergence / breakdown decision,
//                beta, mu = (W^T A W)^-1 (A W)^T r, ring-slot zeroing
//   k_direction4 x += alpha p (the step left by k_update4), then
//                p = r + beta p - U_0 mu_u - W_p mu_p for a tile of lanes;
//                the U_0 rows of a stage arrive in a shared-memory ring by
//                cp.async two stages ahead and serve all the tile's lanes
//   k_update_u0s, k_direction4s  the update (with the shared deflation
//                dots) and the direction with every stream staged through
//                shared memory by cp.async (up to four / two private columns)
//   k_stencil4r, k_stencil4t  z-marching stencil tiles: planes in registers
//                with cp.async halos, or whole planes by TMA tensor copies
//                into a shared-memory ring; the autotuner picks one
//
// Lanes are addressed through the active list `alist` (rebuilt by the host
// at every synchronisation) so converged lanes cost no work; tiles group up
// to 32 active lanes of one sample slot.
#include "common.cuh"

#include <cuda.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

namespace rcg {
namespace {

constexpr int kThreads = 256;
constexpr int TILE = 32;       // lanes per tile
constexpr int UPD_WAVES = 1;   // waves of resident CTAs in a k_update4 launch

__device__ __forceinline__ float dot4(const float4 a, const float4 b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

template <int NV>
__device__ __forceinline__ void block_sum(const float (&acc)[NV], double (&res)[NV]) {
    __shared__ double red[kThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double s = (double)acc[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp][v] = s;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < NV; v += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w][v];
        res[v] = s;
    }
    __syncthreads();
}

// q = A~ p for lane c = alist[blockIdx.y]; 4 consecutive x nodes per thread.
__global__ void __launch_bounds__(kThreads)
k_stencil4(Grid g, const float *__restrict__ D, const float *const *__restrict__ diag_of_col,
           const float *const *__restrict__ src, float *const *__restrict__ dst, const int *__restrict__ alist,
           const int *__restrict__ active, double *__restrict__ dots, unsigned long long *__restrict__ prof) {
    const int c = alist[blockIdx.y];
    if (active[c] == 0) return;
    if (prof && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof, 1ULL);
    const float *__restrict__ x = src[c];
    float *__restrict__ y = dst[c];
    const float *__restrict__ dg = diag_of_col[c];
    const float4 *__restrict__ x4 = (const float4 *)x;
    const float4 *__restrict__ D4 = (const float4 *)D;
    const int nx4 = g.Nx >> 2, sxy = g.Nx * g.Ny, sxy4 = sxy >> 2, nv = (int)(g.n >> 2);
    const bool has_y = g.Ny > 1;
    float acc = 0.f;
    auto node4 = [&](int v) {
        const int p0 = v << 2;
        const int i0 = p0 % g.Nx;
        const int rest = p0 / g.Nx;
        const int j = rest % g.Ny;
        const int k = rest / g.Ny;
        const float4 xc = x4[v], Dc = D4[v], dc = ((const float4 *)dg)[v];
        float4 o = make_float4(dc.x * xc.x, dc.y * xc.y, dc.z * xc.z, dc.w * xc.w);
        // x neighbours inside the row
        const float xl = i0 > 0 ? x[p0 - 1] : 0.f, Dl = i0 > 0 ? D[p0 - 1] : 0.f;
        const float xr = i0 + 4 < g.Nx ? x[p0 + 4] : 0.f, Dr = i0 + 4 < g.Nx ? D[p0 + 4] : 0.f;
        o.x -= (i0 > 0 ? 0.5f * (Dc.x + Dl) * xl : 0.f) + 0.5f * (Dc.x + Dc.y) * xc.y;
        o.y -= 0.5f * (Dc.y + Dc.x) * xc.x + 0.5f * (Dc.y + Dc.z) * xc.z;
        o.z -= 0.5f * (Dc.z + Dc.y) * xc.y + 0.5f * (Dc.z + Dc.w) * xc.w;
        o.w -= 0.5f * (Dc.w + Dc.z) * xc.z + (i0 + 4 < g.Nx ? 0.5f * (Dc.w + Dr) * xr : 0.f);
#define RCG_NB4(cond, off)                                                                     \
        if (cond) {                                                                            \
            const float4 xn = x4[v + (off)], Dn = D4[v + (off)];                               \
            o.x -= 0.5f * (Dc.x + Dn.x) * xn.x; o.y -= 0.5f * (Dc.y + Dn.y) * xn.y;           \
            o.z -= 0.5f * (Dc.z + Dn.z) * xn.z; o.w -= 0.5f * (Dc.w + Dn.w) * xn.w;           \
        }
        RCG_NB4(has_y && j > 0, -nx4)
        RCG_NB4(has_y && j < g.Ny - 1, nx4)
        RCG_NB4(k > 0, -sxy4)
        RCG_NB4(k < g.Nz - 1, sxy4)
#undef RCG_NB4
        ((float4 *)y)[v] = o;
        acc += dot4(xc, o);
    };
    const int stride = gridDim.x * blockDim.x;
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    for (; v + stride < nv; v += 2 * stride) {
        node4(v);
        node4(v + stride);
    }
    if (v < nv) node4(v);
    double s = (double)acc;
    __shared__ double red[kThreads / 32];
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) s += __shfl_down_sync(0xffffffffu, s, o2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        atomicAdd(dots + c, t);
    }
}

// 3D grids with 256 % (Nx / 4) == 0: q = A~ p for ZL lanes per CTA over one
// (y-tile, z-chunk) block.  The CTA's thread (tx, ty) owns x-nodes 4tx..4tx+3
// of row y0 + ty; TY = 256 / (Nx / 4) rows form the tile.  Planes of p (each
// lane) and D, tile rows plus one halo row on either side, stream through a
// ZR-slot shared-memory ring by cp.async two planes ahead, so every p and D
// value is read from memory about once (halo rows and planes aside) and the
// six neighbours come from shared memory.  Fused p^T q per lane.
//
// Every halo a neighbour read can touch holds zeros: a zero pad float4 at
// both ends of each slot row (x ghosts), and the rows and planes outside the
// grid are copied with zero source bytes (y, z ghosts).  A ghost's p is 0, so
// its coupling term vanishes whatever the weight, and the neighbour reads
// need no boundary predicates (the ghosts' share of the diagonal is in the
// precomputed diagonal).
constexpr int ZR = 4;    // ring slots: planes z-1, z, z+1 in use, z+2 in flight
constexpr int ZL = 2;    // lanes per CTA (they share the D planes)

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
}

// Shared-memory bytes of k_stencil4z for an x extent of nx4 float4.
__host__ __device__ constexpr size_t stencil4z_smem(int nx4) {
    return (size_t)ZR * (ZL + 1) * (kThreads / nx4 + 2) * (nx4 + 2) * sizeof(float4);
}

__global__ void __launch_bounds__(kThreads, 3)
k_stencil4z(Grid g, const float *__restrict__ D, const float *const *__restrict__ diag_of_col,
            const float *const *__restrict__ src, float *const *__restrict__ dst, const int *__restrict__ alist,
            int na, const int *__restrict__ active, double *__restrict__ dots, unsigned long long *__restrict__ prof,
            int zc) {
    extern __shared__ float4 ring[];                 // [ZR][ZL + 1][TY + 2][nx4 + 2]
    const int nx4 = g.Nx >> 2, TY = kThreads / nx4, rows = TY + 2, RW = nx4 + 2;
    const int ytiles = (g.Ny + TY - 1) / TY;
    const int yt = blockIdx.x % ytiles, zb = blockIdx.x / ytiles;
    const int y0 = yt * TY, z0 = zb * zc;
    const int z1 = min(z0 + zc, g.Nz);
    const int tx = threadIdx.x % nx4, ty = threadIdx.x / nx4;
    const int y = y0 + ty;
    int c[ZL];
    bool on[ZL];
    int non = 0;
#pragma unroll
    for (int i = 0; i < ZL; ++i) {
        const int li = blockIdx.y * ZL + i;
        c[i] = li < na ? alist[li] : -1;
        on[i] = c[i] >= 0 && active[c[i]] != 0;
        non += on[i];
    }
    if (non == 0 || z0 >= g.Nz) return;             // uniform over the CTA
    if (prof && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof, (unsigned long long)non);
    const float *P[ZL];
    float4 *Q[ZL];
    const float4 *DG[ZL];
#pragma unroll
    for (int i = 0; i < ZL; ++i) {
        P[i] = on[i] ? src[c[i]] : nullptr;
        Q[i] = on[i] ? (float4 *)dst[c[i]] : nullptr;
        DG[i] = on[i] ? (const float4 *)diag_of_col[c[i]] : nullptr;
    }
    const int plane4 = RW * rows;                    // float4 per array and slot
    // slot of plane z (z >= -1)
    auto slot = [&](int z) { return ring + (size_t)((z + ZR) % ZR) * (ZL + 1) * plane4; };
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // zero pads at both ends of every slot row (never written again)
    for (int e = threadIdx.x; e < ZR * (ZL + 1) * rows; e += kThreads) {
        ring[(size_t)e * RW] = zero4;
        ring[(size_t)e * RW + RW - 1] = zero4;
    }
    // Plane z, rows y0-1 .. y0+TY, of each array into its slot; rows and
    // planes outside the grid, and arrays of inactive lanes, as zeros.  Thread
    // (tx, ty) copies column tx of slot rows ty, ty + TY, ... (256 threads =
    // TY rows of nx4 float4), walking (array, row) without division.
    auto load_plane = [&](int z) {
        float4 *sl = slot(z);
        const bool zin = z >= 0 && z < g.Nz;
        int a = 0, ry = ty;
        for (int R = ty; R < (ZL + 1) * rows; R += TY) {
            const int yy = y0 - 1 + ry;
            const float *base = D;
#pragma unroll
            for (int i = 0; i < ZL; ++i)
                if (a == i) base = P[i];
            const bool ok = zin && yy >= 0 && yy < g.Ny && base != nullptr;
            const float4 *s4 = ok ? (const float4 *)base + ((long long)z * g.Ny + yy) * nx4 + tx : (const float4 *)D;
            cp_async16(sl + R * RW + 1 + tx, s4, ok ? 16 : 0);
            ry += TY;
            if (ry >= rows) { ry -= rows; ++a; }
        }
    };
    __syncthreads();                                 // pads before the first cp.async lands beside them
    // prologue: planes z0-1, z0, z0+1 (one cp.async group each)
    for (int q = -1; q <= 1; ++q) {
        if (z0 + q <= z1) load_plane(z0 + q);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const bool yok = y < g.Ny;
    const int row4 = nx4 * g.Ny;                     // float4 per plane in memory
    float4 dgc[ZL], dgn[ZL];
#pragma unroll
    for (int i = 0; i < ZL; ++i)
        dgc[i] = (on[i] && yok) ? DG[i][(long long)z0 * row4 + y * nx4 + tx] : zero4;
    float acc[ZL];
#pragma unroll
    for (int i = 0; i < ZL; ++i) acc[i] = 0.f;
    const int rc = (ty + 1) * RW + 1 + tx, dof = ZL * plane4;
    for (int z = z0; z < z1; ++z) {
        if (z + 2 <= z1) load_plane(z + 2);
        asm volatile("cp.async.commit_group;" ::: "memory");
        const long long v = (long long)z * row4 + y * nx4 + tx;
#pragma unroll
        for (int i = 0; i < ZL; ++i)
            dgn[i] = (on[i] && yok && z + 1 < z1) ? DG[i][v + row4] : zero4;
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        if (yok) {
            const float4 *cs = slot(z), *ms = slot(z - 1), *ps = slot(z + 1);
            const float4 Dc = cs[dof + rc];
            const float Dl = cs[dof + rc - 1].w, Dr = cs[dof + rc + 1].x;
            const float4 Dym = cs[dof + rc - RW], Dyp = cs[dof + rc + RW];
            const float4 Dzm = ms[dof + rc], Dzp = ps[dof + rc];
            // face weights (D_p + D_q) / 2; towards a ghost they meet p = 0
            const float wl = 0.5f * (Dc.x + Dl), wr = 0.5f * (Dc.w + Dr);
            const float w01 = 0.5f * (Dc.x + Dc.y), w12 = 0.5f * (Dc.y + Dc.z), w23 = 0.5f * (Dc.z + Dc.w);
            auto fw = [&](const float4 Dn) {
                return make_float4(0.5f * (Dc.x + Dn.x), 0.5f * (Dc.y + Dn.y), 0.5f * (Dc.z + Dn.z),
                                   0.5f * (Dc.w + Dn.w));
            };
            const float4 wym = fw(Dym), wyp = fw(Dyp), wzm = fw(Dzm), wzp = fw(Dzp);
#pragma unroll
            for (int i = 0; i < ZL; ++i) {
                if (!on[i]) continue;
                const int po = i * plane4;
                const float4 xc = cs[po + rc];
                const float xlv = cs[po + rc - 1].w, xrv = cs[po + rc + 1].x;
                const float4 xym = cs[po + rc - RW], xyp = cs[po + rc + RW];
                const float4 xzm = ms[po + rc], xzp = ps[po + rc];
                const float4 dg = dgc[i];
                float4 o;
                o.x = dg.x * xc.x - (wl * xlv + w01 * xc.y) - (wym.x * xym.x + wyp.x * xyp.x) - (wzm.x * xzm.x + wzp.x * xzp.x);
                o.y = dg.y * xc.y - (w01 * xc.x + w12 * xc.z) - (wym.y * xym.y + wyp.y * xyp.y) - (wzm.y * xzm.y + wzp.y * xzp.y);
                o.z = dg.z * xc.z - (w12 * xc.y + w23 * xc.w) - (wym.z * xym.z + wyp.z * xyp.z) - (wzm.z * xzm.z + wzp.z * xzp.z);
                o.w = dg.w * xc.w - (w23 * xc.z + wr * xrv) - (wym.w * xym.w + wyp.w * xyp.w) - (wzm.w * xzm.w + wzp.w * xzp.w);
                Q[i][v] = o;
                acc[i] += dot4(xc, o);
            }
        }
#pragma unroll
        for (int i = 0; i < ZL; ++i) dgc[i] = dgn[i];
        __syncthreads();                               // slot of plane z-1 is refilled next
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __shared__ double red[kThreads / 32][ZL];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < ZL; ++i) {
        double s = (double)acc[i];
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) s += __shfl_down_sync(0xffffffffu, s, o2);
        if (lane == 0) red[warp][i] = s;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ZL; ++i)
        if (threadIdx.x == i && on[i]) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w][i];
            atomicAdd(dots + c[i], t);
        }
}

// 3D grids with Nx % 4 == 0, any Nx / 4 that TX divides: q = A~ p for ZL
// lanes per CTA over a TX x TY tile of float4 columns (TY = 256 / TX) and a
// chunk of z planes, marching in z.  Thread (tx, ty) owns the float4 column
// (x4 = x0 + tx, y = y0 + ty) and keeps planes z-1, z, z+1 of its own column
// (and z+2 in flight) in registers for every lane and for D, so the two
// z-neighbours cost no shared-memory traffic.  Only the current plane goes
// through shared memory, for the four in-plane neighbours: each thread
// stores its centre value, the edge threads copy the one-cell halo (x and y)
// of the next plane by cp.async (zero-filled outside the grid), one barrier
// per plane, two plane buffers.  D and the sample diagonals are shared by
// the ZL lanes; fused p^T q per lane.
// MB: CTAs per SM the register allocation must allow (2 by default for up to
// two lanes; 3 trades a few spilled registers for occupancy).
template <int TX, int ZL, int MB = (ZL <= 2 ? 2 : 1)>
__global__ void __launch_bounds__(kThreads, MB)
k_stencil4r(Grid g, const float *__restrict__ D, const float *const *__restrict__ diag_of_col,
            const float *const *__restrict__ src, float *const *__restrict__ dst, const int *__restrict__ alist,
            int na, const int *__restrict__ active, double *__restrict__ dots, unsigned long long *__restrict__ prof,
            int zc, int gc) {
    constexpr int TY = kThreads / TX, RW = TX + 2, RH = TY + 2, NA = ZL + 1;
    extern __shared__ float4 pl[];                   // [2][NA][RH][RW]
    const int nx4 = g.Nx >> 2, xtiles = nx4 / TX, ytiles = (g.Ny + TY - 1) / TY;
    // Grid order.  gc > 0: lane groups in chunks of gc, the group within its
    // chunk fastest (blockIdx.x), then the (x tile, y tile, z chunk)
    // (blockIdx.y), then the chunk (blockIdx.z): the CTAs resident together
    // are gc lane groups on a run of tiles, so each tile's D and diagonal
    // planes come from DRAM once per chunk and serve its groups from L2.
    // gc == 0: the tile fastest, then the lane group (each group streams
    // whole planes; D and the diagonal are read again for every group).
    const int lg = gc > 0 ? (int)blockIdx.z * gc + (int)blockIdx.x : (int)blockIdx.y;
    const int tz = gc > 0 ? (int)blockIdx.y : (int)blockIdx.x;
    const int xt = tz % xtiles, rest = tz / xtiles;
    const int yt = rest % ytiles, zb = rest / ytiles;
    const int z0 = zb * zc, z1 = min(z0 + zc, g.Nz);
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x4 = xt * TX + tx, y = yt * TY + ty;
    int c[ZL];
    bool on[ZL];
    int non = 0;
#pragma unroll
    for (int i = 0; i < ZL; ++i) {
        const int li = lg * ZL + i;
        c[i] = li < na ? alist[li] : -1;
        on[i] = c[i] >= 0 && active[c[i]] != 0;
        non += on[i];
    }
    if (non == 0 || z0 >= g.Nz) return;             // uniform over the CTA
    if (prof && tz == 0 && threadIdx.x == 0) atomicAdd(prof, (unsigned long long)non);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 *A[NA];                             // arrays: lanes' p, then D
    float4 *Q[ZL];
    const float4 *DG[ZL];
#pragma unroll
    for (int i = 0; i < ZL; ++i) {
        A[i] = on[i] ? (const float4 *)src[c[i]] : nullptr;
        Q[i] = on[i] ? (float4 *)dst[c[i]] : nullptr;
        DG[i] = on[i] ? (const float4 *)diag_of_col[c[i]] : nullptr;
    }
    A[ZL] = (const float4 *)D;
    // lanes of one sample share the diagonal: load it once for the CTA
    bool shared_dg = on[0];
#pragma unroll
    for (int i = 1; i < ZL; ++i) shared_dg = shared_dg && on[i] && DG[i] == DG[0];
    const bool yok = y < g.Ny;
    const long long row4 = (long long)nx4 * g.Ny;   // float4 per plane
    const long long col = (long long)y * nx4 + x4;  // this thread's column within a plane
    // halo duty: x (tx = 0: x4 - 1, tx = TX - 1: x4 + 1), y (ty = 0: y - 1, ty = TY - 1: y + 1)
    const int hxd = (tx == 0) ? -1 : (tx == TX - 1 ? 1 : 0);
    const int hyd = (ty == 0) ? -1 : (ty == TY - 1 ? 1 : 0);
    const bool hxok = hxd != 0 && yok && x4 + hxd >= 0 && x4 + hxd < nx4;
    const bool hyok = hyd != 0 && y + hyd >= 0 && y + hyd < g.Ny;
    const int cc = (ty + 1) * RW + (tx + 1);        // this thread's cell in a plane buffer
    constexpr int PS = RH * RW;                      // float4 per array and buffer
    auto buf = [&](int z) { return pl + (size_t)(z & 1) * NA * PS; };
    // zero the halo cells no thread fills (corners, and the ghost columns /
    // rows of both buffers are refilled with zero-byte copies below)
    for (int e = threadIdx.x; e < 2 * NA * PS; e += kThreads) pl[e] = zero4;
    __syncthreads();
    // halo cells of plane z into its buffer (cp.async; zero bytes outside the grid)
    auto halo = [&](int z) {
        if (z >= z1) return;                         // plane z1 is only a z-neighbour (registers)
        float4 *b = buf(z);
        const long long pz = (long long)z * row4;
        if (hxd != 0) {
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const bool ok = hxok && A[a] != nullptr;
                cp_async16(b + a * PS + cc + hxd, ok ? A[a] + pz + col + hxd : (const float4 *)D, ok ? 16 : 0);
            }
        }
        if (hyd != 0) {
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const bool ok = hyok && A[a] != nullptr;
                cp_async16(b + a * PS + cc + hyd * RW, ok ? A[a] + pz + col + (long long)hyd * nx4 : (const float4 *)D,
                           ok ? 16 : 0);
            }
        }
    };
    auto ld = [&](int a, int z) -> float4 {
        return (yok && z >= 0 && z < g.Nz && A[a] != nullptr) ? A[a][(long long)z * row4 + col] : zero4;
    };
    float4 pm[NA], pc[NA], pn[NA], pnn[NA], dgc[ZL];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        pm[a] = ld(a, z0 - 1);
        pc[a] = ld(a, z0);
        pn[a] = ld(a, z0 + 1);
    }
#pragma unroll
    for (int i = 0; i < ZL; ++i)
        dgc[i] = (on[i] && yok && (i == 0 || !shared_dg)) ? DG[i][(long long)z0 * row4 + col] : zero4;
    halo(z0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    float acc[ZL];
#pragma unroll
    for (int i = 0; i < ZL; ++i) acc[i] = 0.f;
    for (int z = z0; z < z1; ++z) {
        float4 dgn[ZL];
#pragma unroll
        for (int a = 0; a < NA; ++a) pnn[a] = ld(a, z + 2);
#pragma unroll
        for (int i = 0; i < ZL; ++i)
            dgn[i] = (on[i] && yok && z + 1 < z1 && (i == 0 || !shared_dg)) ? DG[i][(long long)(z + 1) * row4 + col]
                                                                            : zero4;
        float4 *b = buf(z);
#pragma unroll
        for (int a = 0; a < NA; ++a) b[a * PS + cc] = pc[a];
        asm volatile("cp.async.wait_group 0;" ::: "memory");      // this thread's halo copies of plane z
        __syncthreads();                                           // everyone's; plane z-1 reads are done
        halo(z + 1);                                               // into the buffer plane z-1 used
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (yok) {
            const float4 *dp = b + ZL * PS;
            const float4 Dc = pc[ZL];
            const float Dl = dp[cc - 1].w, Dr = dp[cc + 1].x;
            const float4 Dym = dp[cc - RW], Dyp = dp[cc + RW], Dzm = pm[ZL], Dzp = pn[ZL];
            // face weights (D_p + D_q) / 2; towards a ghost they meet p = 0
            const float wl = 0.5f * (Dc.x + Dl), wr = 0.5f * (Dc.w + Dr);
            const float w01 = 0.5f * (Dc.x + Dc.y), w12 = 0.5f * (Dc.y + Dc.z), w23 = 0.5f * (Dc.z + Dc.w);
            auto fw = [&](const float4 Dn) {
                return make_float4(0.5f * (Dc.x + Dn.x), 0.5f * (Dc.y + Dn.y), 0.5f * (Dc.z + Dn.z),
                                   0.5f * (Dc.w + Dn.w));
            };
            const float4 wym = fw(Dym), wyp = fw(Dyp), wzm = fw(Dzm), wzp = fw(Dzp);
            const long long v = (long long)z * row4 + col;
#pragma unroll
            for (int i = 0; i < ZL; ++i) {
                if (!on[i]) continue;
                const float4 *xp = b + i * PS;
                const float4 xc = pc[i];
                const float xlv = xp[cc - 1].w, xrv = xp[cc + 1].x;
                const float4 xym = xp[cc - RW], xyp = xp[cc + RW], xzm = pm[i], xzp = pn[i];
                const float4 dg = shared_dg ? dgc[0] : dgc[i];
                float4 o;
                o.x = dg.x * xc.x - (wl * xlv + w01 * xc.y) - (wym.x * xym.x + wyp.x * xyp.x) - (wzm.x * xzm.x + wzp.x * xzp.x);
                o.y = dg.y * xc.y - (w01 * xc.x + w12 * xc.z) - (wym.y * xym.y + wyp.y * xyp.y) - (wzm.y * xzm.y + wzp.y * xzp.y);
                o.z = dg.z * xc.z - (w12 * xc.y + w23 * xc.w) - (wym.z * xym.z + wyp.z * xyp.z) - (wzm.z * xzm.z + wzp.z * xzp.z);
                o.w = dg.w * xc.w - (w23 * xc.z + wr * xrv) - (wym.w * xym.w + wyp.w * xyp.w) - (wzm.w * xzm.w + wzp.w * xzp.w);
                Q[i][v] = o;
                acc[i] += dot4(xc, o);
            }
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) { pm[a] = pc[a]; pc[a] = pn[a]; pn[a] = pnn[a]; }
#pragma unroll
        for (int i = 0; i < ZL; ++i) dgc[i] = dgn[i];
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __shared__ double red[kThreads / 32][ZL];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < ZL; ++i) {
        double s = (double)acc[i];
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) s += __shfl_down_sync(0xffffffffu, s, o2);
        if (lane == 0) red[warp][i] = s;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ZL; ++i)
        if (threadIdx.x == i && on[i]) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w][i];
            atomicAdd(dots + c[i], t);
        }
}

template <int TX, int ZL>
constexpr size_t stencil4r_smem() {
    return (size_t)2 * (ZL + 1) * (kThreads / TX + 2) * (TX + 2) * sizeof(float4);
}

// r -= alpha q; r^T r and the private (A W)^T r dots (the shared ones come
// from k_u0dots) for the active lanes alist[0 .. na-1].  The step
// x += alpha p is left to k_direction4 of the same iteration, which reads p
// anyway: alpha and the iteration number go to xa / xt.
// The work is flattened: lane li has nb units of kThreads float4, and CTA c
// takes the contiguous units [U c / G, U (c+1) / G) of the U = na nb units
// (G = gridDim.x, one wave of resident CTAs), so every CTA moves the same
// bytes whatever na is.  The dots of each lane segment a CTA crosses are
// summed in the CTA and added atomically; the CTA that holds a lane's first
// unit does the lane's one-off work.  KPM bounds the lanes' private columns;
// a thread loads UNR float4 of every stream before it uses any (the loads in
// flight per SM are what bounds this kernel).
template <int KPM>
__host__ __device__ constexpr int upd_unroll() { return KPM <= 2 ? 4 : KPM <= 4 ? 2 : 1; }

template <int KPM>
__global__ void __launch_bounds__(kThreads, 2)
k_update4(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ alist, int na, int t, int sprev,
          int scur, int spq, int sw) {
    constexpr int NV = 1 + KPM;
    constexpr int UNR = upd_unroll<KPM>();
    __shared__ double out[NV];
    const long long nv = n >> 2;
    const long long nb = (nv + kThreads - 1) / kThreads;
    const long long U = (long long)na * nb;
    const long long u_end = U * (blockIdx.x + 1) / gridDim.x;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long u = U * blockIdx.x / gridDim.x; u < u_end;) {
        const int li = (int)(u / nb);
        const long long lane0 = (long long)li * nb;
        const long long seg_end = u_end < lane0 + nb ? u_end : lane0 + nb;
        const bool owner = u == lane0;
        const int l = alist[li];
        const long long v0 = (u - lane0) * kThreads, v1 = (seg_end - lane0) * kThreads;
        u = seg_end;
        if (ls.active[l] == 0) continue;
        const double pq = ls.pq[spq * ls.m + l];
        const double rrp = ls.rr[sprev * ls.m + l];
        if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rrp)) {
            if (owner && threadIdx.x == 0) ls.flag[l] = 2;
            continue;
        }
        const float alpha = (float)(rrp / pq);
        const int ku = gm.k_u, kp = gm.kp[l];
        if (owner && threadIdx.x == 0) {
            ls.xa[l] = alpha;
            ls.xt[l] = t;
            ls.pq[(1 - spq) * ls.m + l] = 0.0;
            if (ls.prof) { atomicAdd(ls.prof + 1, 1ULL); atomicAdd(ls.prof + 2, (unsigned long long)(ku + kp)); }
        }
        float acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = 0.f;
        const long long o = (long long)l * gm.ld;
        float4 *__restrict__ R = (float4 *)((float *)gm.r + o);
        const float4 *__restrict__ Q = (const float4 *)((const float *)gm.q + o);
        const float *__restrict__ AP = (const float *)gm.awp + (long long)l * gm.kp_max * gm.ld;
        const long long vend = v1 < nv ? v1 : nv;
        for (long long v = v0 + threadIdx.x; v < vend; v += (long long)UNR * kThreads) {
            float4 qv[UNR], rv[UNR], av[UNR][KPM];
#pragma unroll
            for (int e = 0; e < UNR; ++e) {
                const long long w = v + (long long)e * kThreads;
                const bool ok = w < vend;
                qv[e] = ok ? Q[w] : z4;
                rv[e] = ok ? R[w] : z4;
#pragma unroll
                for (int c = 0; c < KPM; ++c)
                    av[e][c] = (ok && c < kp) ? ((const float4 *)(AP + (long long)c * gm.ld))[w] : z4;
            }
#pragma unroll
            for (int e = 0; e < UNR; ++e) {
                const long long w = v + (long long)e * kThreads;
                const float4 r1 = make_float4(rv[e].x - alpha * qv[e].x, rv[e].y - alpha * qv[e].y,
                                              rv[e].z - alpha * qv[e].z, rv[e].w - alpha * qv[e].w);
                if (w < vend) R[w] = r1;
                acc[0] += dot4(r1, r1);
#pragma unroll
                for (int c = 0; c < KPM; ++c) acc[1 + c] += dot4(av[e][c], r1);
            }
        }
        block_sum<NV>(acc, out);
        if (threadIdx.x == 0) atomicAdd(ls.rr + scur * ls.m + l, out[0]);
        if (threadIdx.x >= 1 && threadIdx.x <= kp)
            atomicAdd(ls.wv + ((long long)sw * ls.m + l) * KMAX + ku + (threadIdx.x - 1), out[threadIdx.x]);
    }
}

// One wave of resident k_update4<KPM> CTAs for lanes with at most KPM
// private columns (occupancy cached per device ordinal).
template <int KPM>
void launch_update4(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const LaneList &ll,
                    int t, int sprev, int scur, int spq, int sw) {
    static int slots[64] = {};
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    int g = 2 * 152;
    if (dev >= 0 && dev < 64) {
        if (!slots[dev]) {
            int occ = 0, sms = 0;
            RCG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_update4<KPM>, kThreads, 0));
            RCG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            slots[dev] = std::max(1, occ * sms);
        }
        g = slots[dev];
    }
    const long long units = (long long)ll.na * (((n >> 2) + kThreads - 1) / kThreads);
    const int grid = (int)std::min<long long>(units, (long long)UPD_WAVES * g);
    k_update4<KPM><<<grid, kThreads, 0, st>>>(n, gm, ls, ll.alist, ll.na, t, sprev, scur, spq, sw);
}

// wv[sw][l][c] += (A~_s U_0)_c^T r_l (use_w: U_0 itself) for the lanes of
// tile blockIdx.y (one sample slot) over this CTA's node range.  The range is
// walked in stages of SN nodes: the r rows of the tile's lanes (32 x SN) and
// the k_u x SN block of A~_s U_0 stream into a U0_NST-slot shared-memory ring
// by cp.async, two stages ahead.  Thread (warp w, lane slot l) dots float4
// nodes 4w..4w+3 of the stage of lane l against every column (the column
// reads are warp-wide broadcasts); the eight warps' partial sums are added in
// shared memory at the end.
constexpr int SN = 128;                 // nodes per stage
constexpr int SN4 = SN / 4;
constexpr int RP = SN4 + 1;             // padded float4 stride of an r row (conflict-free reads)
constexpr int U0_NST = 3;
constexpr int DIR_NST = 3;              // U_0 stage ring of k_direction4
template <int KUT>
__host__ __device__ constexpr int u0_stage4() { return TILE * RP + KUT * SN4; }
template <int KUT>
constexpr size_t u0_smem() { return (size_t)U0_NST * u0_stage4<KUT>() * sizeof(float4); }

template <int KUT>
__global__ void __launch_bounds__(kThreads)
k_u0dots(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ tile_lane, const int *__restrict__ tile_si,
         const int *__restrict__ tile_cnt, int sw, long long chunk, int use_w) {
    extern __shared__ float4 u0s[];
    __shared__ int lanes[TILE];
    constexpr int STG = u0_stage4<KUT>();
    const int t = blockIdx.y;
    const int cnt = tile_cnt[t], ku = gm.k_u;
    if (threadIdx.x < TILE) lanes[threadIdx.x] = threadIdx.x < cnt ? tile_lane[t * TILE + threadIdx.x] : -1;
    const float *__restrict__ AU =
        use_w ? (const float *)gm.wu : (const float *)gm.awu + (long long)tile_si[t] * ku * gm.ld;
    const float *__restrict__ Rb = (const float *)gm.r;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    const int nst = r1 > r0 ? (int)((r1 - r0 + SN - 1) / SN) : 0;
    __syncthreads();
    // this thread's copies: r rows (lane e/SN4, float4 e%SN4) and U_0 rows
    auto issue = [&](int s) {
        float4 *stg = u0s + (size_t)(s % U0_NST) * STG;
        const long long base = r0 + (long long)s * SN;
        for (int e = threadIdx.x; e < TILE * SN4; e += kThreads) {
            const int l = e / SN4, v4 = e % SN4;
            const long long p = base + 4 * v4;
            const int ln = lanes[l];
            const bool ok = ln >= 0 && p < r1;
            const float *src = ok ? Rb + (long long)ln * gm.ld + p : Rb;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(stg + l * RP + v4)),
                         "l"(src), "r"(ok ? 16 : 0)
                         : "memory");
        }
        for (int e = threadIdx.x; e < KUT * SN4; e += kThreads) {
            const int c = e / SN4, v4 = e % SN4;
            const long long p = base + 4 * v4;
            const bool ok = c < ku && p < r1;
            const float *src = ok ? AU + (long long)c * gm.ld + p : AU;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(stg + TILE * RP + e)),
                         "l"(src), "r"(ok ? 16 : 0)
                         : "memory");
        }
    };
    const int warp = threadIdx.x >> 5, tl = threadIdx.x & 31;
    float acc[KUT], acc2[KUT];                     // lanes tl mod 16 and tl mod 16 + 16
#pragma unroll
    for (int c = 0; c < KUT; ++c) { acc[c] = 0.f; acc2[c] = 0.f; }
    for (int q = 0; q < 2; ++q) {
        if (q < nst) issue(q);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int s = 0; s < nst; ++s) {
        if (s + 2 < nst) issue(s + 2);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 2;" ::: "memory");
        __syncthreads();
        {
            // thread (warp w, tl): lanes la = tl mod 16 and la + 16, float4 4w + 2 (tl / 16) + {0, 1};
            // each U_0 float4 read serves both lanes
            const float4 *stg = u0s + (size_t)(s % U0_NST) * STG;
            const int la = tl & 15, vb = warp * 4 + 2 * (tl >> 4);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int v4 = vb + j;
                const float4 r0 = stg[la * RP + v4], r1 = stg[(la + 16) * RP + v4];
#pragma unroll
                for (int c = 0; c < KUT; ++c) {
                    const float4 u = stg[TILE * RP + c * SN4 + v4];
                    acc[c] = fmaf(u.x, r0.x, fmaf(u.y, r0.y, fmaf(u.z, r0.z, fmaf(u.w, r0.w, acc[c]))));
                    acc2[c] = fmaf(u.x, r1.x, fmaf(u.y, r1.y, fmaf(u.z, r1.z, fmaf(u.w, r1.w, acc2[c]))));
                }
            }
        }
        __syncthreads();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // sum the partials: red[h][w][c][l], h = half-warp (tl / 16), lane l = tl mod 16 (+16 for acc2)
    float *red = (float *)u0s;
    const int h = tl >> 4, la = tl & 15;
#pragma unroll
    for (int c = 0; c < KUT; ++c) {
        red[((h * (kThreads / 32) + warp) * KUT + c) * TILE + la] = acc[c];
        red[((h * (kThreads / 32) + warp) * KUT + c) * TILE + la + 16] = acc2[c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < KUT * TILE; e += kThreads) {
        const int c = e / TILE, l = e % TILE;
        if (l < cnt && c < ku) {
            float v = 0.f;
#pragma unroll
            for (int w = 0; w < 2 * (kThreads / 32); ++w) v += red[(w * KUT + c) * TILE + l];
            atomicAdd(ls.wv + ((long long)sw * ls.m + lanes[l]) * KMAX + c, (double)v);
        }
    }
}

// The update and the shared deflation dots in one pass over r, for the
// lanes of tile blockIdx.y (<= 32 lanes of one sample slot) over this CTA's
// node range: r -= alpha q; rr += r^T r; wv[c] += (A~_s U_0)_c^T r (c < k_u,
// the U_0 images staged per stage of SN nodes in a cp.async ring and shared
// by the tile's lanes); wv[k_u + c] += (A~ W_p)_c^T r (private columns).
// It replaces k_update4 + k_u0dots inside an iteration: r is read once
// instead of twice.  512 threads: thread (warp w, tl) serves lanes w + 16 q
// (q < 2), float4 tl of every stage; the loads of both lanes go out before
// their use (two lanes' accumulators per thread keep the registers below the
// 128 of one 512-thread CTA per SM).  The CTA
// with blockIdx.x == 0 records each lane's step (xa, xt) and clears the next
// p^T q slot, as the owner CTA of k_update4 does.
constexpr int kUU = 512;                // threads of k_update_u0
int device_sms(int dev);                 // SMs of a device (cached)
template <int KUT, int KPM>
__global__ void __launch_bounds__(kUU, 1)
k_update_u0(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ tile_lane, const int *__restrict__ tile_si,
            const int *__restrict__ tile_cnt, int t, int sprev, int scur, int spq, int sw, long long chunk) {
    constexpr int NV = 1 + KUT + KPM;
    constexpr int NL = TILE / (kUU / 32);     // lanes per thread (2)
    constexpr int G = KPM <= 4 ? 2 : 1;
    __shared__ float4 Us[U0_NST][KUT][SN4];
    __shared__ int slane[TILE], skp[TILE];
    __shared__ float salpha[TILE];
    const int tt = blockIdx.y, cnt = tile_cnt[tt], ku = gm.k_u;
    if (threadIdx.x < TILE) {
        int l = threadIdx.x < cnt ? tile_lane[tt * TILE + threadIdx.x] : -1;
        float a = 0.f;
        if (l >= 0 && ls.active[l] != 0) {
            const double pq = ls.pq[spq * ls.m + l], rrp = ls.rr[sprev * ls.m + l];
            if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rrp)) {
                if (blockIdx.x == 0) ls.flag[l] = 2;          // breakdown: every CTA skips the lane
                l = -1;
            } else {
                a = (float)(rrp / pq);
                if (blockIdx.x == 0) {
                    ls.xa[l] = a;
                    ls.xt[l] = t;
                    ls.pq[(1 - spq) * ls.m + l] = 0.0;
                    if (ls.prof) {
                        atomicAdd(ls.prof + 1, 1ULL);
                        atomicAdd(ls.prof + 2, (unsigned long long)(ku + gm.kp[l]));
                    }
                }
            }
        } else {
            l = -1;
        }
        slane[threadIdx.x] = l;
        salpha[threadIdx.x] = a;
        skp[threadIdx.x] = l >= 0 ? gm.kp[l] : 0;
    }
    const float *__restrict__ AU = (const float *)gm.awu + (long long)tile_si[tt] * ku * gm.ld;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    const int nst = r1 > r0 ? (int)((r1 - r0 + SN - 1) / SN) : 0;
    __syncthreads();
    auto issue = [&](int st) {
        if (st < nst) {
            const long long base = r0 + (long long)st * SN;
            for (int e = threadIdx.x; e < KUT * SN4; e += kUU) {
                const int c = e / SN4, v4 = e % SN4;
                const long long p = base + 4 * v4;
                const bool ok = c < ku && p < r1;
                const float *src = ok ? AU + (long long)c * gm.ld + p : AU;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                                 (uint32_t)__cvta_generic_to_shared(&Us[st % U0_NST][c][v4])),
                             "l"(src), "r"(ok ? 16 : 0)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int warp = threadIdx.x >> 5, tl = threadIdx.x & 31;
    float acc[NL][NV];
#pragma unroll
    for (int q = 0; q < NL; ++q)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[q][v] = 0.f;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    issue(0);
    issue(1);
    for (int st = 0; st < nst; ++st) {
        issue(st + 2);
        asm volatile("cp.async.wait_group 2;" ::: "memory");     // stage st: this thread's copies
        __syncthreads();                                          // ... and everyone's
        const long long p = r0 + (long long)st * SN + 4 * tl;
        if (p < r1) {
#pragma unroll
            for (int q0 = 0; q0 < NL; q0 += G) {
                float4 qv[G], rv[G], av[G][KPM];
#pragma unroll
                for (int gq = 0; gq < G; ++gq) {
                    const int l = slane[warp + (kUU / 32) * (q0 + gq)];
                    const long long o = (long long)(l < 0 ? 0 : l) * gm.ld + p;
                    qv[gq] = l >= 0 ? *(const float4 *)((const float *)gm.q + o) : z4;
                    rv[gq] = l >= 0 ? *(const float4 *)((const float *)gm.r + o) : z4;
                    const int kp = skp[warp + (kUU / 32) * (q0 + gq)];
                    const float *AP = (const float *)gm.awp + (long long)(l < 0 ? 0 : l) * gm.kp_max * gm.ld + p;
#pragma unroll
                    for (int c = 0; c < KPM; ++c)
                        av[gq][c] = (l >= 0 && c < kp) ? *(const float4 *)(AP + (long long)c * gm.ld) : z4;
                }
#pragma unroll
                for (int gq = 0; gq < G; ++gq) {
                    const int jj = warp + (kUU / 32) * (q0 + gq);
                    const int l = slane[jj];
                    if (l < 0) continue;
                    const float a = salpha[jj];
                    const float4 rn = make_float4(rv[gq].x - a * qv[gq].x, rv[gq].y - a * qv[gq].y,
                                                  rv[gq].z - a * qv[gq].z, rv[gq].w - a * qv[gq].w);
                    *(float4 *)((float *)gm.r + (long long)l * gm.ld + p) = rn;
                    float *ac = acc[q0 + gq];
                    ac[0] += dot4(rn, rn);
#pragma unroll
                    for (int c = 0; c < KUT; ++c) ac[1 + c] += dot4(Us[st % U0_NST][c][tl], rn);
#pragma unroll
                    for (int c = 0; c < KPM; ++c) ac[1 + KUT + c] += dot4(av[gq][c], rn);
                }
            }
        }
        __syncthreads();                                          // the ring slot of stage st is refilled next
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // warp sums per lane, one atomic per lane and column
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        const int jj = warp + (kUU / 32) * q;
        const int l = slane[jj];
        if (l < 0) continue;                                      // uniform over the warp
        const int kp = skp[jj];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            float x = acc[q][v];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (tl == 0) {
                if (v == 0) atomicAdd(ls.rr + scur * ls.m + l, (double)x);
                else if (v <= KUT) {
                    if (v - 1 < ku) atomicAdd(ls.wv + ((long long)sw * ls.m + l) * KMAX + (v - 1), (double)x);
                } else if (v - 1 - KUT < kp) {
                    atomicAdd(ls.wv + ((long long)sw * ls.m + l) * KMAX + ku + (v - 1 - KUT), (double)x);
                }
            }
        }
    }
}

// k_update_u0 with every stream staged through shared memory: each thread
// copies its own float4 of r, q and the private A~W columns of its two lanes
// by cp.async into a ring of NST stages (its own data: no barrier needed for
// it), NST - 1 stages ahead of its use, next to the tile's shared A~_s U_0
// rows.  The register version keeps one stage of loads in flight per thread
// (124 registers, one 512-thread CTA per SM: ~68% of the DRAM bandwidth);
// here NST - 1 stages are in flight in shared memory.  Same arithmetic,
// same reductions.
template <int KPM>
__host__ __device__ constexpr int uus_nst() { return KPM <= 1 ? 4 : KPM <= 2 ? 3 : 2; }
template <int KUT, int KPM>
constexpr size_t uus_smem() {
    return sizeof(float4) * (size_t)uus_nst<KPM>() * (KUT * SN4 + 2 * (2 + KPM) * kUU);
}

template <int KUT, int KPM>
__global__ void __launch_bounds__(kUU, 1)
k_update_u0s(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ tile_lane, const int *__restrict__ tile_si,
             const int *__restrict__ tile_cnt, int t, int sprev, int scur, int spq, int sw, long long chunk) {
    constexpr int NST = uus_nst<KPM>();
    constexpr int NV = 1 + KUT + KPM;
    constexpr int NW = kUU / 32;              // warps
    constexpr int NL = TILE / NW;             // lanes per thread (2)
    constexpr int NB = 2 + KPM;               // r, q, private columns
    extern __shared__ float4 usm[];
    float4 *Us = usm;                         // [NST][KUT][SN4]
    float4 *Ls = usm + NST * KUT * SN4;       // [NST][NL][NB][kUU]
    __shared__ int slane[TILE], skp[TILE];
    __shared__ float salpha[TILE];
    const int tt = blockIdx.x, cnt = tile_cnt[tt], ku = gm.k_u;   // tiles fastest: resident CTAs share A~U_0 rows in L2
    if (threadIdx.x < TILE) {
        int l = threadIdx.x < cnt ? tile_lane[tt * TILE + threadIdx.x] : -1;
        float a = 0.f;
        if (l >= 0 && ls.active[l] != 0) {
            const double pq = ls.pq[spq * ls.m + l], rrp = ls.rr[sprev * ls.m + l];
            if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rrp)) {
                if (blockIdx.y == 0) ls.flag[l] = 2;          // breakdown: every CTA skips the lane
                l = -1;
            } else {
                a = (float)(rrp / pq);
                if (blockIdx.y == 0) {
                    ls.xa[l] = a;
                    ls.xt[l] = t;
                    ls.pq[(1 - spq) * ls.m + l] = 0.0;
                    if (ls.prof) {
                        atomicAdd(ls.prof + 1, 1ULL);
                        atomicAdd(ls.prof + 2, (unsigned long long)(ku + gm.kp[l]));
                    }
                }
            }
        } else {
            l = -1;
        }
        slane[threadIdx.x] = l;
        salpha[threadIdx.x] = a;
        skp[threadIdx.x] = l >= 0 ? gm.kp[l] : 0;
    }
    const float *__restrict__ AU = (const float *)gm.awu + (long long)tile_si[tt] * ku * gm.ld;
    const long long r0 = (long long)blockIdx.y * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    const int nst = r1 > r0 ? (int)((r1 - r0 + SN - 1) / SN) : 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, tl = threadIdx.x & 31;
    int myl[NL], mykp[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        myl[q] = slane[warp + NW * q];
        mykp[q] = skp[warp + NW * q];
    }
    const float *Rb = (const float *)gm.r, *Qb = (const float *)gm.q, *Wb = (const float *)gm.awp;
    auto cp16 = [](float4 *dst, const float *src, bool ok) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                     "l"(src), "r"(ok ? 16 : 0)
                     : "memory");
    };
    auto issue = [&](int st) {
        if (st < nst) {
            const long long base = r0 + (long long)st * SN;
            const int slot = st % NST;
            for (int e = threadIdx.x; e < KUT * SN4; e += kUU) {
                const int c = e / SN4, v4 = e % SN4;
                const long long p = base + 4 * v4;
                const bool ok = c < ku && p < r1;
                cp16(&Us[(slot * KUT + c) * SN4 + v4], ok ? AU + (long long)c * gm.ld + p : AU, ok);
            }
            const long long p = base + 4 * tl;
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                const int l = myl[q];
                const bool okp = l >= 0 && p < r1;
                const long long o = (long long)(l < 0 ? 0 : l) * gm.ld + p;
                float4 *dst = Ls + ((slot * NL + q) * NB) * kUU + threadIdx.x;
                cp16(dst, okp ? Rb + o : Rb, okp);
                cp16(dst + kUU, okp ? Qb + o : Qb, okp);
                const float *AP = Wb + (long long)(l < 0 ? 0 : l) * gm.kp_max * gm.ld + p;
#pragma unroll
                for (int c = 0; c < KPM; ++c) {
                    const bool ok = okp && c < mykp[q];
                    cp16(dst + (2 + c) * kUU, ok ? AP + (long long)c * gm.ld : Rb, ok);
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float acc[NL][NV];
#pragma unroll
    for (int q = 0; q < NL; ++q)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[q][v] = 0.f;
#pragma unroll
    for (int st = 0; st < NST - 1; ++st) issue(st);
    for (int st = 0; st < nst; ++st) {
        issue(st + NST - 1);
        asm volatile("cp.async.wait_group %0;" ::"n"(NST - 1) : "memory");   // stage st: this thread's copies
        __syncthreads();                                                   // ... and the U_0 rows of all threads
        const int slot = st % NST;
        const long long p = r0 + (long long)st * SN + 4 * tl;
        if (p < r1) {
            float4 rn[NL];
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                const int l = myl[q];
                rn[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (l < 0) continue;
                const float4 *src = Ls + ((slot * NL + q) * NB) * kUU + threadIdx.x;
                const float4 rv = src[0], qv = src[kUU];
                const float a = salpha[warp + NW * q];
                rn[q] = make_float4(rv.x - a * qv.x, rv.y - a * qv.y, rv.z - a * qv.z, rv.w - a * qv.w);
                *(float4 *)((float *)gm.r + (long long)l * gm.ld + p) = rn[q];
                float *ac = acc[q];
                ac[0] += dot4(rn[q], rn[q]);
#pragma unroll
                for (int c = 0; c < KPM; ++c) ac[1 + KUT + c] += dot4(src[(2 + c) * kUU], rn[q]);
            }
            // each U_0 row once for both lanes (an absent lane's rn is zero)
#pragma unroll
            for (int c = 0; c < KUT; ++c) {
                const float4 u = Us[(slot * KUT + c) * SN4 + tl];
#pragma unroll
                for (int q = 0; q < NL; ++q) acc[q][1 + c] += dot4(u, rn[q]);
            }
        }
        __syncthreads();                                          // the U_0 slot of stage st is refilled next
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        const int l = myl[q];
        if (l < 0) continue;                                      // uniform over the warp
        const int kp = mykp[q];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            float x = acc[q][v];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (tl == 0) {
                if (v == 0) atomicAdd(ls.rr + scur * ls.m + l, (double)x);
                else if (v <= KUT) {
                    if (v - 1 < ku) atomicAdd(ls.wv + ((long long)sw * ls.m + l) * KMAX + (v - 1), (double)x);
                } else if (v - 1 - KUT < kp) {
                    atomicAdd(ls.wv + ((long long)sw * ls.m + l) * KMAX + ku + (v - 1 - KUT), (double)x);
                }
            }
        }
    }
}

template <int KUT, int KPM>
void launch_update_u0s(cudaStream_t st, dim3 grid, long long n, LaneGeom gm, LaneState ls, const LaneList &ll, int t,
                       int sprev, int scur, int spq, int sw, long long chunk) {
    static bool attr[64] = {};
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_update_u0s<KUT, KPM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)uus_smem<KUT, KPM>()));
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    k_update_u0s<KUT, KPM><<<dim3(grid.y, grid.x), kUU, uus_smem<KUT, KPM>(), st>>>(
        n, gm, ls, ll.tile_lane, ll.tile_si, ll.tile_cnt, t, sprev, scur, spq, sw, chunk);
}

template <int KUT>
void u0dots_attr() {
    static bool attr[64] = {};
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_u0dots<KUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)u0_smem<KUT>()));
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
}

// One warp per lane l = alist[blockIdx.x]: decision, beta, mu (float), slot zeroing.
__global__ void __launch_bounds__(32)
k_mu(LaneState ls, const int *__restrict__ alist, int sprev, int scur, int snext, int sw, float *__restrict__ mu,
     float *__restrict__ beta, int restart) {
    const int l = alist[blockIdx.x];
    if (ls.active[l] == 0) return;
    const double rc = ls.rr[scur * ls.m + l];
    const bool broke = (ls.flag[l] == 2) || !isfinite(rc);
    const bool conv = !broke && sqrt(rc) <= ls.thresh[l];
    __syncwarp();
    if (threadIdx.x == 0) {
        if (!restart) ls.iters[l] += 1;
        if (broke) { ls.active[l] = 0; ls.flag[l] = 2; }
        else if (conv) { ls.active[l] = 0; ls.flag[l] = 1; }
        ls.rr[snext * ls.m + l] = 0.0;
        if (ls.prof && !restart && !broke && !conv) { atomicAdd(ls.prof + 3, 1ULL); atomicAdd(ls.prof + 4, (unsigned long long)ls.kdef[l]); }
    }
    if (broke || conv) {
        for (int c = threadIdx.x; c < KMAX; c += 32) ls.wv[((long long)(1 - sw) * ls.m + l) * KMAX + c] = 0.0;
        return;
    }
    const int k = ls.kdef[l];
    const double *G = ls.gw + (long long)l * KMAX * KMAX;
    const double *w = ls.wv + ((long long)sw * ls.m + l) * KMAX;
    for (int i = threadIdx.x; i < k; i += 32) {
        double s = 0.0;
        for (int jj = 0; jj < k; ++jj) s += G[i + jj * KMAX] * w[jj];
        mu[(long long)l * KMAX + i] = (float)s;
    }
    if (threadIdx.x == 0) beta[l] = restart ? 0.f : (float)(rc / ls.rr[sprev * ls.m + l]);
    __syncwarp();
    for (int c = threadIdx.x; c < KMAX; c += 32) ls.wv[((long long)(1 - sw) * ls.m + l) * KMAX + c] = 0.0;
}

// Iteration it over the lanes of tile blockIdx.y and this CTA's node range:
// x += alpha p (the step k_update4 left, for every lane whose xt is it, also
// one that stopped in this iteration), then, for the active lanes,
// p = r + beta p - U_0 mu_u - W_p mu_p.  U_0 is staged per stage of SN nodes
// in a shared-memory ring and shared by the tile's lanes (warp w: lanes
// w + 8q); one barrier per stage.
template <int KUT, int KPM>
__global__ void __launch_bounds__(kThreads, 2)
k_direction4(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ tile_lane,
             const int *__restrict__ tile_cnt, const float *__restrict__ mu, const float *__restrict__ beta,
             long long chunk, int it) {
    __shared__ float4 Us[DIR_NST][KUT][SN / 4];
    __shared__ float smu[TILE][KU_MAX + KP_MAX];
    __shared__ float sbeta[TILE], salpha[TILE];
    __shared__ int slane[TILE], skp[TILE], sdir[TILE];
    __shared__ const float *spw[TILE][KPM];
    const int t = blockIdx.y, cnt = tile_cnt[t], ku = gm.k_u;
    if (threadIdx.x < TILE) {
        int l = threadIdx.x < cnt ? tile_lane[t * TILE + threadIdx.x] : -1;
        const bool step = l >= 0 && ls.xt[l] == it;
        const bool dir = l >= 0 && ls.active[l] != 0;
        if (!step && !dir) l = -1;
        slane[threadIdx.x] = l;
        sdir[threadIdx.x] = dir ? 1 : 0;
        salpha[threadIdx.x] = step ? ls.xa[l] : 0.f;
        skp[threadIdx.x] = dir ? gm.kp[l] : 0;
        sbeta[threadIdx.x] = dir ? beta[l] : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TILE * (KU_MAX + KP_MAX); e += blockDim.x) {
        const int jj = e / (KU_MAX + KP_MAX), c = e % (KU_MAX + KP_MAX);
        const int l = slane[jj];
        smu[jj][c] = (l >= 0 && sdir[jj] && c < ku + skp[jj]) ? mu[(long long)l * KMAX + c] : 0.f;
    }
    for (int e = threadIdx.x; e < TILE * KPM; e += blockDim.x) {
        const int jj = e / KPM, c = e % KPM;
        const int l = slane[jj];
        spw[jj][c] = (l >= 0 && sdir[jj] && c < skp[jj]) ? (const float *)gm.wpp[(long long)l * KPT + c] : nullptr;
    }
    const int warp = threadIdx.x >> 5, tl = threadIdx.x & 31;
    const float *__restrict__ WU = (const float *)gm.wu;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    const int nst = r1 > r0 ? (int)((r1 - r0 + SN - 1) / SN) : 0;
    // U_0 rows of stage st into ring slot st % DIR_NST (cp.async, one group per
    // stage; rows past r1 and columns past k_u are zeros written directly)
    auto stage_u = [&](int st) {
        if (st < nst) {
            const long long base = r0 + (long long)st * SN;
            for (int e = threadIdx.x; e < KUT * (SN / 4); e += blockDim.x) {
                const int c = e / (SN / 4), v4 = e % (SN / 4);
                const long long p = base + 4 * v4;
                float4 *dst = &Us[st % DIR_NST][c][v4];
                if (c < ku && p < r1)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                                     (uint32_t)__cvta_generic_to_shared(dst)),
                                 "l"(WU + (long long)c * gm.ld + p)
                                 : "memory");
                else
                    *dst = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    stage_u(0);
    stage_u(1);
    for (int st = 0; st < nst; ++st) {
        const long long base = r0 + (long long)st * SN;
        asm volatile("cp.async.wait_group 1;" ::: "memory");      // stage st: this thread's copies
        __syncthreads();                                           // everyone's; stage st-1 is done
        stage_u(st + 2);                                           // into the slot stage st-1 used
        const float4(&Uc)[KUT][SN / 4] = Us[st % DIR_NST];
        const long long p = base + 4 * tl;
        if (p < r1) {
            // the loads of G lanes before any of their stores (a store to one
            // lane's p or x would otherwise hold back the next lane's loads)
            constexpr int G = KPM <= 2 ? 4 : KPM <= 4 ? 2 : 1;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int q0 = 0; q0 < 4; q0 += G) {
                float4 pv[G], xv[G], rv[G], wv[G][KPM];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int jj = warp + 8 * (q0 + g);
                    const int l = slane[jj];
                    const bool dir = l >= 0 && sdir[jj] != 0;
                    const long long o = (long long)(l < 0 ? 0 : l) * gm.ld + p;
                    pv[g] = l >= 0 ? *(const float4 *)((const float *)gm.p + o) : z4;
                    xv[g] = (l >= 0 && salpha[jj] != 0.f) ? *(const float4 *)((const float *)gm.x + o) : z4;
                    rv[g] = dir ? *(const float4 *)((const float *)gm.r + o) : z4;
                    const int kp = skp[jj];
#pragma unroll
                    for (int c = 0; c < KPM; ++c)
                        wv[g][c] = (dir && c < kp) ? *(const float4 *)(spw[jj][c] + p) : z4;
                }
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int jj = warp + 8 * (q0 + g);
                    const int l = slane[jj];
                    if (l < 0) continue;
                    const long long o = (long long)l * gm.ld + p;
                    const float a = salpha[jj];
                    if (a != 0.f)
                        *(float4 *)((float *)gm.x + o) = make_float4(xv[g].x + a * pv[g].x, xv[g].y + a * pv[g].y,
                                                                     xv[g].z + a * pv[g].z, xv[g].w + a * pv[g].w);
                    if (!sdir[jj]) continue;
                    const float b = sbeta[jj];
                    float4 sres = make_float4(rv[g].x + b * pv[g].x, rv[g].y + b * pv[g].y, rv[g].z + b * pv[g].z,
                                              rv[g].w + b * pv[g].w);
#pragma unroll
                    for (int c = 0; c < KUT; ++c) {
                        const float m = c < ku ? smu[jj][c] : 0.f;
                        const float4 u = Uc[c][tl];
                        sres.x -= m * u.x; sres.y -= m * u.y; sres.z -= m * u.z; sres.w -= m * u.w;
                    }
                    const int kp = skp[jj];
#pragma unroll
                    for (int c = 0; c < KPM; ++c) {
                        if (c >= kp) break;
                        const float m = smu[jj][ku + c];
                        sres.x -= m * wv[g][c].x; sres.y -= m * wv[g][c].y;
                        sres.z -= m * wv[g][c].z; sres.w -= m * wv[g][c].w;
                    }
                    *(float4 *)((float *)gm.p + o) = sres;
                }
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// k_direction4s: k_direction4 with every stream staged through shared
// memory, as k_update_u0s does for the update: 512 threads, each thread
// serves two lanes of the tile (lanes w and w + 16 of warp w) and copies its
// own float4 of p, x (lanes that take the step), r and the private W
// columns of both lanes by cp.async into a ring of NST stages, NST - 1
// stages ahead of their use, next to the tile's U_0 rows.  The register
// version keeps one batch of loads per warp in flight and drains it at
// every stage barrier (16 warps per SM at 128 registers: ~73% of the DRAM
// bandwidth on the 64^3 bench step).  Same arithmetic.
template <int KPM>
__host__ __device__ constexpr int dirs_nst() { return KPM <= 1 ? 3 : 2; }
template <int KUT, int KPM>
constexpr size_t dirs_smem() {
    return sizeof(float4) * (size_t)dirs_nst<KPM>() * (KUT * SN4 + 2 * (3 + KPM) * kUU);
}

template <int KUT, int KPM>
__global__ void __launch_bounds__(kUU, 1)
k_direction4s(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ tile_lane,
              const int *__restrict__ tile_cnt, const float *__restrict__ mu, const float *__restrict__ beta,
              long long chunk, int it) {
    constexpr int NST = dirs_nst<KPM>();
    constexpr int NW = kUU / 32;              // warps
    constexpr int NL = TILE / NW;             // lanes per thread (2)
    constexpr int NB = 3 + KPM;               // p, x, r, private columns
    extern __shared__ float4 dsm[];
    float4 *Us = dsm;                         // [NST][KUT][SN4]
    float4 *Ls = dsm + NST * KUT * SN4;       // [NST][NL][NB][kUU]
    __shared__ float smu[TILE][KU_MAX + KP_MAX];
    __shared__ float sbeta[TILE], salpha[TILE];
    __shared__ int slane[TILE], skp[TILE], sdir[TILE];
    __shared__ const float *spw[TILE][KPM];
    const int t = blockIdx.x, cnt = tile_cnt[t], ku = gm.k_u;     // tiles fastest: resident CTAs share U_0 rows in L2
    if (threadIdx.x < TILE) {
        int l = threadIdx.x < cnt ? tile_lane[t * TILE + threadIdx.x] : -1;
        const bool step = l >= 0 && ls.xt[l] == it;
        const bool dir = l >= 0 && ls.active[l] != 0;
        if (!step && !dir) l = -1;
        slane[threadIdx.x] = l;
        sdir[threadIdx.x] = dir ? 1 : 0;
        salpha[threadIdx.x] = step ? ls.xa[l] : 0.f;
        skp[threadIdx.x] = dir ? gm.kp[l] : 0;
        sbeta[threadIdx.x] = dir ? beta[l] : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TILE * (KU_MAX + KP_MAX); e += blockDim.x) {
        const int jj = e / (KU_MAX + KP_MAX), c = e % (KU_MAX + KP_MAX);
        const int l = slane[jj];
        smu[jj][c] = (l >= 0 && sdir[jj] && c < ku + skp[jj]) ? mu[(long long)l * KMAX + c] : 0.f;
    }
    for (int e = threadIdx.x; e < TILE * KPM; e += blockDim.x) {
        const int jj = e / KPM, c = e % KPM;
        const int l = slane[jj];
        spw[jj][c] = (l >= 0 && sdir[jj] && c < skp[jj]) ? (const float *)gm.wpp[(long long)l * KPT + c] : nullptr;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, tl = threadIdx.x & 31;
    int myl[NL], myj[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        myj[q] = warp + NW * q;
        myl[q] = slane[myj[q]];
    }
    const float *__restrict__ WU = (const float *)gm.wu;
    const float *Pb = (const float *)gm.p, *Xb = (const float *)gm.x, *Rb = (const float *)gm.r;
    const long long r0 = (long long)blockIdx.y * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    const int nst = r1 > r0 ? (int)((r1 - r0 + SN - 1) / SN) : 0;
    auto cp16 = [](float4 *dst, const float *src, bool ok) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                     "l"(src), "r"(ok ? 16 : 0)
                     : "memory");
    };
    auto issue = [&](int st) {
        if (st < nst) {
            const long long base = r0 + (long long)st * SN;
            const int slot = st % NST;
            for (int e = threadIdx.x; e < KUT * SN4; e += kUU) {
                const int c = e / SN4, v4 = e % SN4;
                const long long p = base + 4 * v4;
                const bool ok = c < ku && p < r1;
                cp16(&Us[(slot * KUT + c) * SN4 + v4], ok ? WU + (long long)c * gm.ld + p : WU, ok);
            }
            const long long p = base + 4 * tl;
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                const int l = myl[q], jj = myj[q];
                const bool okp = l >= 0 && p < r1;
                const bool dir = okp && sdir[jj] != 0;
                const long long o = (long long)(l < 0 ? 0 : l) * gm.ld + p;
                float4 *dst = Ls + ((slot * NL + q) * NB) * kUU + threadIdx.x;
                cp16(dst, okp ? Pb + o : Pb, okp);
                cp16(dst + kUU, (okp && salpha[jj] != 0.f) ? Xb + o : Xb, okp && salpha[jj] != 0.f);
                cp16(dst + 2 * kUU, dir ? Rb + o : Rb, dir);
#pragma unroll
                for (int c = 0; c < KPM; ++c) {
                    const bool ok = dir && c < skp[jj];
                    cp16(dst + (3 + c) * kUU, ok ? spw[jj][c] + p : Rb, ok);
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int st = 0; st < NST - 1; ++st) issue(st);
    for (int st = 0; st < nst; ++st) {
        issue(st + NST - 1);
        asm volatile("cp.async.wait_group %0;" ::"n"(NST - 1) : "memory");   // stage st: this thread's copies
        __syncthreads();                                                   // ... and the U_0 rows of all threads
        const int slot = st % NST;
        const long long p = r0 + (long long)st * SN + 4 * tl;
        if (p < r1) {
            float4 sres[NL];
            bool dq[NL];
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                const int l = myl[q], jj = myj[q];
                sres[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                dq[q] = l >= 0 && sdir[jj] != 0;
                if (l < 0) continue;
                const float4 *src = Ls + ((slot * NL + q) * NB) * kUU + threadIdx.x;
                const float4 pv = src[0];
                const float a = salpha[jj];
                if (a != 0.f) {
                    const float4 xv = src[kUU];
                    *(float4 *)((float *)gm.x + (long long)l * gm.ld + p) =
                        make_float4(xv.x + a * pv.x, xv.y + a * pv.y, xv.z + a * pv.z, xv.w + a * pv.w);
                }
                if (!dq[q]) continue;
                const float4 rv = src[2 * kUU];
                const float b = sbeta[jj];
                sres[q] = make_float4(rv.x + b * pv.x, rv.y + b * pv.y, rv.z + b * pv.z, rv.w + b * pv.w);
            }
            // each U_0 row once for both lanes
#pragma unroll
            for (int c = 0; c < KUT; ++c) {
                const float4 u = Us[(slot * KUT + c) * SN4 + tl];
#pragma unroll
                for (int q = 0; q < NL; ++q) {
                    const float m = (c < ku && dq[q]) ? smu[myj[q]][c] : 0.f;
                    sres[q].x -= m * u.x; sres[q].y -= m * u.y; sres[q].z -= m * u.z; sres[q].w -= m * u.w;
                }
            }
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                if (!dq[q]) continue;
                const int jj = myj[q], kp = skp[jj];
                const float4 *src = Ls + ((slot * NL + q) * NB) * kUU + threadIdx.x;
#pragma unroll
                for (int c = 0; c < KPM; ++c) {
                    if (c >= kp) break;
                    const float m = smu[jj][ku + c];
                    const float4 w = src[(3 + c) * kUU];
                    sres[q].x -= m * w.x; sres[q].y -= m * w.y; sres[q].z -= m * w.z; sres[q].w -= m * w.w;
                }
                *(float4 *)((float *)gm.p + (long long)myl[q] * gm.ld + p) = sres[q];
            }
        }
        __syncthreads();                                          // stage st's slot is refilled next
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int KUT, int KPM>
void dir_launch_s(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const LaneList &ll,
                  const float *mu, const float *beta, int it) {
    static bool attr[64] = {};
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_direction4s<KUT, KPM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)dirs_smem<KUT, KPM>()));
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    // node ranges (multiples of SN) for ~4 waves of one CTA per SM over the tiles
    long long z = std::max<long long>(1, 4LL * device_sms(dev) / std::max(ll.ntiles, 1));
    const long long maxz = (n + 4 * SN - 1) / (4 * SN);
    if (z > maxz) z = maxz;
    long long chunk = (n + z - 1) / z;
    chunk = (chunk + SN - 1) / SN * SN;
    z = (n + chunk - 1) / chunk;
    k_direction4s<KUT, KPM><<<dim3(ll.ntiles, (unsigned)z), kUU, dirs_smem<KUT, KPM>(), st>>>(
        n, gm, ls, ll.tile_lane, ll.tile_cnt, mu, beta, chunk, it);
}

// k_direction4<KUT, KPM> over the tiles of ll in one wave of resident CTAs
// (occupancy cached per device ordinal): a partial second wave would hold
// the whole launch.  Node ranges are multiples of SN.
template <int KUT, int KPM>
void dir_launch(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const LaneList &ll,
                const float *mu, const float *beta, int it) {
    static int slots[64] = {};
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    int sl = 2 * 152;
    if (dev >= 0 && dev < 64) {
        if (!slots[dev]) {
            int occ = 0, sms = 0;
            RCG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_direction4<KUT, KPM>, kThreads, 0));
            RCG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            slots[dev] = std::max(1, occ * sms);
        }
        sl = slots[dev];
    }
    long long z = std::max<long long>(1, sl / std::max(ll.ntiles, 1));
    const long long maxz = (n + 4 * SN - 1) / (4 * SN);
    if (z > maxz) z = maxz;
    long long chunk = (n + z - 1) / z;
    chunk = (chunk + SN - 1) / SN * SN;
    z = (n + chunk - 1) / chunk;
    k_direction4<KUT, KPM><<<dim3((unsigned)z, ll.ntiles), kThreads, 0, st>>>(n, gm, ls, ll.tile_lane, ll.tile_cnt,
                                                                             mu, beta, chunk, it);
}

template <int KUT>
void dir_launch_kp(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const LaneList &ll,
                   const float *mu, const float *beta, int it) {
    // up to two private columns: the staged kernel; more: the register version
    if (gm.kp_sel <= 1) dir_launch_s<KUT, 1>(st, n, gm, ls, ll, mu, beta, it);
    else if (gm.kp_sel <= 2) dir_launch_s<KUT, 2>(st, n, gm, ls, ll, mu, beta, it);
    else if (gm.kp_sel <= 4) dir_launch<KUT, 4>(st, n, gm, ls, ll, mu, beta, it);
    else dir_launch<KUT, KP_MAX>(st, n, gm, ls, ll, mu, beta, it);
}

void direction_launch(cudaStream_t st, int kut, long long n, const LaneGeom &gm, const LaneState &ls,
                      const LaneList &ll, const float *mu, const float *beta, int it) {
    switch (kut) {
        case 0: case 4: dir_launch_kp<4>(st, n, gm, ls, ll, mu, beta, it); break;
        case 8: dir_launch_kp<8>(st, n, gm, ls, ll, mu, beta, it); break;
        case 12: dir_launch_kp<12>(st, n, gm, ls, ll, mu, beta, it); break;
        default: dir_launch_kp<16>(st, n, gm, ls, ll, mu, beta, it);
    }
}

// Lane l = alist[blockIdx.y]: wv[sw][k_u + c] += (src_c)^T r over the lane's
// private columns (src = W or A W) and optionally rr[srr] += r^T r.
__global__ void __launch_bounds__(kThreads)
k_private_dots4(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ alist, int use_aw, int sw,
                int with_rr, int srr) {
    const int l = alist[blockIdx.y];
    const int ku = gm.k_u, kp = gm.kp[l];
    if (kp == 0 && !with_rr) return;
    constexpr int NV = 1 + KP_MAX;
    float acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.f;
    const float4 *__restrict__ R = (const float4 *)((const float *)gm.r + (long long)l * gm.ld);
    const float *S[KP_MAX];
#pragma unroll
    for (int c = 0; c < KP_MAX; ++c)
        S[c] = c >= kp ? nullptr
                       : use_aw ? (const float *)gm.awp + ((long long)l * gm.kp_max + c) * gm.ld
                                : (const float *)gm.wpp[(long long)l * KPT + c];
    const int nv = (int)(n >> 2);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        const float4 rv = R[v];
        acc[0] += dot4(rv, rv);
#pragma unroll
        for (int c = 0; c < KP_MAX; ++c)
            if (c < kp) acc[1 + c] += dot4(((const float4 *)S[c])[v], rv);
    }
    __shared__ double out[NV];
    block_sum<NV>(acc, out);
    if (threadIdx.x == 0 && with_rr) atomicAdd(ls.rr + srr * ls.m + l, out[0]);
    if (threadIdx.x >= 1 && threadIdx.x <= kp)
        atomicAdd(ls.wv + ((long long)sw * ls.m + l) * KMAX + ku + (threadIdx.x - 1), out[threadIdx.x]);
}

// One warp per lane l = alist[blockIdx.x]: mu = Ginv * wv[sw] (float), no decision.
__global__ void __launch_bounds__(32)
k_mu_only(LaneState ls, const int *__restrict__ alist, int sw, float *__restrict__ mu) {
    const int l = alist[blockIdx.x];
    const int k = ls.kdef[l];
    const double *G = ls.gw + (long long)l * KMAX * KMAX;
    const double *w = ls.wv + ((long long)sw * ls.m + l) * KMAX;
    for (int i = threadIdx.x; i < k; i += 32) {
        double s = 0.0;
        for (int jj = 0; jj < k; ++jj) s += G[i + jj * KMAX] * w[jj];
        mu[(long long)l * KMAX + i] = (float)s;
    }
}

// Restart projection of the lanes of tile blockIdx.y (one sample slot):
// x = U_0 mu_u + W_p mu_p;  r -= A~_s U_0 mu_u + A~_s W_p mu_p.
template <int KUT>
__global__ void __launch_bounds__(kThreads)
k_project4(long long n, LaneGeom gm, const int *__restrict__ tile_lane, const int *__restrict__ tile_si,
           const int *__restrict__ tile_cnt, const float *__restrict__ mu, long long chunk) {
    __shared__ float4 Us[KUT][SN / 4], As_[KUT][SN / 4];
    __shared__ float smu[TILE][KU_MAX + KP_MAX];
    __shared__ int slane[TILE], skp[TILE];
    const int t = blockIdx.y, cnt = tile_cnt[t], ku = gm.k_u;
    if (threadIdx.x < TILE) {
        const int l = threadIdx.x < cnt ? tile_lane[t * TILE + threadIdx.x] : -1;
        slane[threadIdx.x] = l;
        skp[threadIdx.x] = l >= 0 ? gm.kp[l] : 0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TILE * (KU_MAX + KP_MAX); e += blockDim.x) {
        const int jj = e / (KU_MAX + KP_MAX), c = e % (KU_MAX + KP_MAX);
        const int l = slane[jj];
        smu[jj][c] = (l >= 0 && c < ku + skp[jj]) ? mu[(long long)l * KMAX + c] : 0.f;
    }
    const float *__restrict__ WU = (const float *)gm.wu;
    const float *__restrict__ AU = (const float *)gm.awu + (long long)tile_si[t] * ku * gm.ld;
    const int warp = threadIdx.x >> 5, tl = threadIdx.x & 31;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    __syncthreads();
    for (long long base = r0; base < r1; base += SN) {
        for (int e = threadIdx.x; e < KUT * (SN / 4); e += blockDim.x) {
            const int c = e / (SN / 4), v4 = e % (SN / 4);
            const long long p = base + 4 * v4;
            const bool ok = c < ku && p < r1;
            Us[c][v4] = ok ? *(const float4 *)(WU + (long long)c * gm.ld + p) : make_float4(0.f, 0.f, 0.f, 0.f);
            As_[c][v4] = ok ? *(const float4 *)(AU + (long long)c * gm.ld + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const long long p = base + 4 * tl;
        if (p < r1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int jj = warp + 8 * q;
                const int l = slane[jj];
                if (l < 0) continue;
                float4 xs = make_float4(0.f, 0.f, 0.f, 0.f), rs = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int c = 0; c < KUT; ++c) {
                    const float m = c < ku ? smu[jj][c] : 0.f;
                    const float4 u = Us[c][tl], a = As_[c][tl];
                    xs.x += m * u.x; xs.y += m * u.y; xs.z += m * u.z; xs.w += m * u.w;
                    rs.x += m * a.x; rs.y += m * a.y; rs.z += m * a.z; rs.w += m * a.w;
                }
                const int kp = skp[jj];
                const float *AP = (const float *)gm.awp + (long long)l * gm.kp_max * gm.ld;
                for (int c = 0; c < kp; ++c) {
                    const float m = smu[jj][ku + c];
                    const float4 w = *(const float4 *)((const float *)gm.wpp[(long long)l * KPT + c] + p);
                    const float4 a = *(const float4 *)(AP + (long long)c * gm.ld + p);
                    xs.x += m * w.x; xs.y += m * w.y; xs.z += m * w.z; xs.w += m * w.w;
                    rs.x += m * a.x; rs.y += m * a.y; rs.z += m * a.z; rs.w += m * a.w;
                }
                const long long o = (long long)l * gm.ld + p;
                *(float4 *)((float *)gm.x + o) = xs;
                float4 rv = *(const float4 *)((const float *)gm.r + o);
                rv.x -= rs.x; rv.y -= rs.y; rv.z -= rs.z; rv.w -= rs.w;
                *(float4 *)((float *)gm.r + o) = rv;
            }
        }
        __syncthreads();
    }
}

int gx_for(long long nv, int rows, int per_sm) {
    long long want = ((long long)per_sm * 152 + rows - 1) / rows;
    long long maxb = (nv + kThreads - 1) / kThreads;
    long long gx = want < maxb ? want : maxb;
    return (int)(gx < 1 ? 1 : gx);
}

}  // namespace

bool cg4_supported(const Grid &g) { return (g.Nx % 4) == 0 && (g.ld % 4) == 0; }

// The plane-streaming stencil: 3D, whole rows of float4 tiling 256 threads.
bool stencil4z_supported(const Grid &g) {
    const int nx4 = g.Nx / 4;
    return g.Ny > 1 && (g.Nx % 4) == 0 && nx4 >= 1 && nx4 <= kThreads && kThreads % nx4 == 0 &&
           stencil4z_smem(nx4) <= 160 * 1024 && g.n < (1LL << 31);
}

namespace {

int device_sms(int dev) {
    static int sms[64] = {};
    if (dev < 0 || dev >= 64) return 152;
    if (!sms[dev]) {
        int v = 0;
        RCG_CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
        sms[dev] = v > 0 ? v : 152;
    }
    return sms[dev];
}

// k_stencil4r<TX, ZL> over the lanes of ll: per-plane tiles x lane groups x
// z-chunks, the chunks sized for ~4 waves of resident CTAs (>= 8 planes each).
// gc: lane groups per chunk of the grid order (see k_stencil4r); -1 (the
// variants' choice) puts all groups in one chunk for up to 16 groups and
// takes the tile-first order above that.
template <int TX, int ZL, int MB = (ZL <= 2 ? 2 : 1)>
void launch_s4r(cudaStream_t st, const Grid &g, const float *D, const float *const *diag, const float *const *p,
                float *const *q, const LaneList &ll, const int *active, double *dots, unsigned long long *prof,
                int gc = -1) {
    static int occ[64] = {};
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    const size_t smem = stencil4r_smem<TX, ZL>();
    if (dev < 0 || dev >= 64 || !occ[dev]) {
        RCG_CUDA_TRY(
            cudaFuncSetAttribute(k_stencil4r<TX, ZL, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int o = 0;
        RCG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_stencil4r<TX, ZL, MB>, kThreads, smem));
        if (dev >= 0 && dev < 64) occ[dev] = std::max(o, 1);
    }
    const int o = (dev >= 0 && dev < 64) ? occ[dev] : 1;
    const int nx4 = g.Nx / 4, TY = kThreads / TX;
    const long long T = (long long)(nx4 / TX) * ((g.Ny + TY - 1) / TY), G = (ll.na + ZL - 1) / ZL;
    const long long resident = (long long)o * device_sms(dev);
    long long nzc = (4 * resident + T * G - 1) / (T * G);
    const long long maxc = std::max<long long>(1, g.Nz / 8);
    nzc = std::max<long long>(1, std::min(nzc, maxc));
    const int zc = (int)((g.Nz + nzc - 1) / nzc);
    nzc = (g.Nz + zc - 1) / zc;
    if (gc < 0) gc = G <= 16 ? (int)G : 0;
    if (gc > G) gc = (int)G;
    const long long nchunk = gc > 0 ? (G + gc - 1) / gc : 0;
    if ((gc > 0 ? std::max(T * nzc, nchunk) : G) > 65535) throw Error{RCG_ERR_INVALID, "k_stencil4r: grid extent"};
    const dim3 grid = gc > 0 ? dim3((unsigned)gc, (unsigned)(T * nzc), (unsigned)nchunk)
                             : dim3((unsigned)(T * nzc), (unsigned)G);
    k_stencil4r<TX, ZL, MB><<<grid, kThreads, smem, st>>>(g, D, diag, p, q, ll.alist, ll.na, active, dots, prof, zc,
                                                          gc);
}

void launch_s4z(cudaStream_t st, const Grid &g, const float *D, const float *const *diag, const float *const *p,
                float *const *q, const LaneList &ll, const int *active, double *dots, unsigned long long *prof) {
    const int nx4 = g.Nx / 4, TY = kThreads / nx4;
    const int ytiles = (g.Ny + TY - 1) / TY, pairs = (ll.na + ZL - 1) / ZL;
    // z-chunks: enough CTAs for ~4 waves at 3 CTAs per SM, chunks of >= 4 planes
    const long long base = (long long)ytiles * pairs;
    long long nzc = (12LL * 152 + base - 1) / base;
    const long long maxc = (g.Nz + 3) / 4;
    if (nzc > maxc) nzc = maxc;
    if (nzc < 1) nzc = 1;
    const int zc = (int)((g.Nz + nzc - 1) / nzc);
    nzc = (g.Nz + zc - 1) / zc;
    const size_t smem = stencil4z_smem(nx4);
    static bool attr[64] = {};
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_stencil4z, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    k_stencil4z<<<dim3((unsigned)(ytiles * nzc), pairs), kThreads, smem, st>>>(g, D, diag, p, q, ll.alist, ll.na,
                                                                               active, dots, prof, zc);
}

// ---------------------------------------------------------------- TMA stencil
// k_stencil4t<ZL, TY>: q = A~ p for ZL lanes per CTA over a tile of 64 x TY
// nodes (x, y), marching in z over a chunk of planes.  Every plane of the
// tile (with a one-node halo in y, four floats in x so that the copy starts
// on a 16-byte boundary) arrives in shared memory by one TMA tensor copy per
// array (the lanes' p, D, and the lanes' sample diagonals without halo) on a
// ring of US4 stages with an mbarrier each; the copy of plane z + 3 is issued
// as soon as plane z - 1's stage is free, so two planes per CTA are in
// flight without holding registers.  Out-of-grid planes and rows arrive as
// zeros (the Dirichlet ghosts; the Robin faces are in the diagonal).  Thread
// (tx, ty) computes the float4 column x = 4 tx of row ty for every lane from
// shared memory, stores q and adds p^T q.  Every mbarrier wait is bounded:
// on timeout the CTA records the error in g_s4t_err, waits (bounded) for the
// copies it issued and returns.
constexpr int US4 = 4;                  // stages of the plane ring
constexpr int T4X = 64;                 // tile width in nodes (16 float4 columns)
constexpr int T4W = T4X + 8;            // copied row width: x0 - 4 .. x0 + 67
constexpr long long S4T_SPIN = 1LL << 22;
__device__ int g_s4t_err;

__host__ __device__ constexpr int s4t_align(int b) { return (b + 127) / 128 * 128; }
template <int TY> __host__ __device__ constexpr int s4t_pbox() { return s4t_align(T4W * (TY + 2) * 4); }
template <int TY> __host__ __device__ constexpr int s4t_gbox() { return s4t_align(T4X * TY * 4); }
template <int ZL, int TY> __host__ __device__ constexpr int s4t_stage() {
    return (ZL + 1) * s4t_pbox<TY>() + ZL * s4t_gbox<TY>();
}
template <int ZL, int TY> constexpr size_t s4t_smem() { return (size_t)US4 * s4t_stage<ZL, TY>() + 1024; }

__device__ __forceinline__ uint32_t s4_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool s4_try_wait(uint32_t mbar, uint32_t parity) {
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

__device__ __forceinline__ void tma4(uint32_t dst, const CUtensorMap *tm, int x, int y, int z, int w, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"((unsigned long long)tm), "r"(x), "r"(y), "r"(z), "r"(w), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tma3(uint32_t dst, const CUtensorMap *tm, int x, int y, int z, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"((unsigned long long)tm), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}

template <int ZL, int TY>
__global__ void __launch_bounds__(16 * TY)
k_stencil4t(const __grid_constant__ CUtensorMap tm_p, const __grid_constant__ CUtensorMap tm_d,
            const __grid_constant__ CUtensorMap tm_g, Grid g, const float *gbase,
            const float *const *__restrict__ diag_of_col, float *const *__restrict__ dst,
            const int *__restrict__ alist, int na, const int *__restrict__ active, double *__restrict__ dots,
            unsigned long long *__restrict__ prof, int zc) {
    constexpr int NT = 16 * TY, PB = s4t_pbox<TY>(), GB = s4t_gbox<TY>(), SB = s4t_stage<ZL, TY>();
    extern __shared__ __align__(1024) char s4t_raw[];
    __shared__ __align__(8) unsigned long long mbar[US4];
    __shared__ int s_ok;
    char *sm = (char *)(((uintptr_t)s4t_raw + 1023) & ~(uintptr_t)1023);
    const int xtiles = g.Nx / T4X, ytiles = (g.Ny + TY - 1) / TY;
    const int tz = blockIdx.x, lg = blockIdx.y;
    const int xt = tz % xtiles, rest = tz / xtiles, yt = rest % ytiles, zb = rest / ytiles;
    const int z0 = zb * zc, z1 = min(z0 + zc, g.Nz);
    int c[ZL], slot[ZL];
    bool on[ZL];
    int non = 0;
#pragma unroll
    for (int i = 0; i < ZL; ++i) {
        const int li = lg * ZL + i;
        c[i] = li < na ? alist[li] : -1;
        on[i] = c[i] >= 0 && active[c[i]] != 0;
        slot[i] = on[i] ? (int)((diag_of_col[c[i]] - gbase) / g.ld) : 0;
        non += on[i];
    }
    if (non == 0 || z0 >= g.Nz) return;                // uniform over the CTA
    if (prof && tz == 0 && threadIdx.x == 0) atomicAdd(prof, (unsigned long long)non);
    const int x0 = xt * T4X, y0 = yt * TY;
    // bytes of one plane's copies (the lanes that are on, D, their diagonals)
    const uint32_t tx_bytes = (uint32_t)(non * (T4W * (TY + 2) * 4 + T4X * TY * 4) + T4W * (TY + 2) * 4);
    if (threadIdx.x == 0) {
        for (int s = 0; s < US4; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s4_u32(&mbar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_ok = 1;
    }
    __syncthreads();
    // plane j of the ring = grid plane z0 - 1 + j, in stage j mod US4; planes
    // z0 - 1 .. z1 are needed
    const int nplanes = z1 - z0 + 2;
    auto issue = [&](int j) {                           // thread 0 only
        const int z = z0 - 1 + j;
        char *st = sm + (j % US4) * SB;
        const uint32_t mb = s4_u32(&mbar[j % US4]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(tx_bytes) : "memory");
#pragma unroll
        for (int i = 0; i < ZL; ++i)
            if (on[i]) {
                tma4(s4_u32(st + i * PB), &tm_p, x0 - 4, y0 - 1, z, c[i], mb);
                tma4(s4_u32(st + (ZL + 1) * PB + i * GB), &tm_g, x0, y0, z, slot[i], mb);
            }
        tma3(s4_u32(st + ZL * PB), &tm_d, x0 - 4, y0 - 1, z, mb);
    };
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int j = 0; j < US4 && j < nplanes; ++j) issue(j);
    }
    int issued = min(US4, nplanes);                      // planes thread 0 issued (the same count in every thread)
    int waited = 0;                                      // planes waited for
    auto wait_plane = [&](int j) -> bool {
        const uint32_t mb = s4_u32(&mbar[j % US4]);
        const uint32_t par = (uint32_t)((j / US4) & 1);
        for (long long it = 0; it < S4T_SPIN; ++it)
            if (s4_try_wait(mb, par)) return true;
        return false;
    };
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int y = y0 + ty, x4 = (x0 >> 2) + tx;
    const bool yok = y < g.Ny;
    const long long row4 = (long long)(g.Nx >> 2) * g.Ny;
    const int cc = (ty + 1) * T4W + 4 + 4 * tx;          // this thread's first float in a p or D box
    const int gc4 = ty * T4X + 4 * tx;                   // ... in a diagonal box
    float acc[ZL];
#pragma unroll
    for (int i = 0; i < ZL; ++i) acc[i] = 0.f;
    bool ok = true;
    // planes z0 - 1 and z0 before the first step; every thread leaves with
    // the same verdict (the steps below hold barriers)
    for (; waited < 2 && waited < nplanes; ++waited)
        if (!wait_plane(waited)) s_ok = 0;
    __syncthreads();
    if (!s_ok) ok = false;
    for (int z = z0; z < z1 && ok; ++z) {
        const int jz = z - z0 + 1;                      // ring index of plane z
        if (!wait_plane(jz + 1)) { ok = false; s_ok = 0; }
        waited = jz + 2;
        __syncthreads();
        if (!s_ok) { ok = false; break; }
        if (yok) {
            const char *sm_m = sm + ((jz - 1) % US4) * SB, *sm_c = sm + (jz % US4) * SB,
                       *sm_p = sm + ((jz + 1) % US4) * SB;
            const float *Dc_ = (const float *)(sm_c + ZL * PB);
            const float4 Dc = *(const float4 *)(Dc_ + cc);
            const float Dl = Dc_[cc - 1], Dr = Dc_[cc + 4];
            const float4 Dym = *(const float4 *)(Dc_ + cc - T4W), Dyp = *(const float4 *)(Dc_ + cc + T4W);
            const float4 Dzm = *(const float4 *)((const float *)(sm_m + ZL * PB) + cc);
            const float4 Dzp = *(const float4 *)((const float *)(sm_p + ZL * PB) + cc);
            const float wl = 0.5f * (Dc.x + Dl), wr = 0.5f * (Dc.w + Dr);
            const float w01 = 0.5f * (Dc.x + Dc.y), w12 = 0.5f * (Dc.y + Dc.z), w23 = 0.5f * (Dc.z + Dc.w);
            auto fw = [&](const float4 Dn) {
                return make_float4(0.5f * (Dc.x + Dn.x), 0.5f * (Dc.y + Dn.y), 0.5f * (Dc.z + Dn.z),
                                   0.5f * (Dc.w + Dn.w));
            };
            const float4 wym = fw(Dym), wyp = fw(Dyp), wzm = fw(Dzm), wzp = fw(Dzp);
            const long long v = (long long)z * row4 + (long long)y * (g.Nx >> 2) + x4;
#pragma unroll
            for (int i = 0; i < ZL; ++i) {
                if (!on[i]) continue;
                const float *P = (const float *)(sm_c + i * PB);
                const float4 xc = *(const float4 *)(P + cc);
                const float xlv = P[cc - 1], xrv = P[cc + 4];
                const float4 xym = *(const float4 *)(P + cc - T4W), xyp = *(const float4 *)(P + cc + T4W);
                const float4 xzm = *(const float4 *)((const float *)(sm_m + i * PB) + cc);
                const float4 xzp = *(const float4 *)((const float *)(sm_p + i * PB) + cc);
                const float4 dg = *(const float4 *)((const float *)(sm_c + (ZL + 1) * PB + i * GB) + gc4);
                float4 o;
                o.x = dg.x * xc.x - (wl * xlv + w01 * xc.y) - (wym.x * xym.x + wyp.x * xyp.x) - (wzm.x * xzm.x + wzp.x * xzp.x);
                o.y = dg.y * xc.y - (w01 * xc.x + w12 * xc.z) - (wym.y * xym.y + wyp.y * xyp.y) - (wzm.y * xzm.y + wzp.y * xzp.y);
                o.z = dg.z * xc.z - (w12 * xc.y + w23 * xc.w) - (wym.z * xym.z + wyp.z * xyp.z) - (wzm.z * xzm.z + wzp.z * xzp.z);
                o.w = dg.w * xc.w - (w23 * xc.z + wr * xrv) - (wym.w * xym.w + wyp.w * xyp.w) - (wzm.w * xzm.w + wzp.w * xzp.w);
                ((float4 *)dst[c[i]])[v] = o;
                acc[i] += dot4(xc, o);
            }
        }
        __syncthreads();                                 // plane z - 1's stage is free
        if (threadIdx.x == 0 && jz - 1 + US4 < nplanes) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(jz - 1 + US4);
        }
        if (jz - 1 + US4 < nplanes) issued = jz + US4;
    }
    // no copy may land in the CTA's shared memory after it exits: wait for
    // every issued plane not yet waited for (the normal path has none left)
    for (int j = waited; j < issued; ++j) wait_plane(j);
    if (!ok && threadIdx.x == 0) atomicExch(&g_s4t_err, RCG_ERR_TIMEOUT);
    __shared__ double red[NT / 32][ZL];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < ZL; ++i) {
        double sacc = (double)acc[i];
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o2);
        if (lane == 0) red[warp][i] = sacc;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ZL; ++i)
        if (threadIdx.x == i && on[i] && ok) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += red[w][i];
            atomicAdd(dots + c[i], t);
        }
}

// cuTensorMapEncodeTiled from the driver, through the runtime (no link
// against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    });
    return fn;
}

// A float32 tensor map of rank r (dims[0] fastest, strides in bytes of
// dims 1..r-1) with the given box; zero fill outside.
void make_map(CUtensorMap *m, const float *base, int r, const cuuint64_t *dims, const cuuint64_t *strides,
              const cuuint32_t *box) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) throw Error{RCG_ERR_CUDA, "cuTensorMapEncodeTiled is not available"};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const CUresult rc = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)r, (void *)base, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rc != CUDA_SUCCESS) throw Error{RCG_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)rc) + ")"};
}

bool s4t_supported(const Grid &g) {
    return cg4_supported(g) && g.Ny > 1 && g.Nx % T4X == 0 && g.Nx <= 4096 && g.n < (1LL << 31);
}

bool s4t_usable(const Grid &g, const LaneList &ll) {
    return s4t_supported(g) && ll.pbase && ll.gbase && ll.pcols > 0 && ll.gslots > 0 && ((uintptr_t)ll.pbase & 15) == 0 &&
           ((uintptr_t)ll.gbase & 15) == 0 && ll.pld % 4 == 0 && g.ld % 4 == 0;
}

template <int ZL, int TY>
void launch_s4t(cudaStream_t st, const Grid &g, const float *D, const float *const *diag, float *const *q,
                const LaneList &ll, const int *active, double *dots, unsigned long long *prof) {
    if (!s4t_usable(g, ll)) throw Error{RCG_ERR_INVALID, "k_stencil4t: lane layout unknown"};
    CUtensorMap tp, td, tg;
    const cuuint64_t sx = (cuuint64_t)g.Nx * 4, sxy = sx * (cuuint64_t)g.Ny, sxyz = sxy * (cuuint64_t)g.Nz;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)g.Nx, (cuuint64_t)g.Ny, (cuuint64_t)g.Nz, (cuuint64_t)ll.pcols};
        const cuuint64_t strides[3] = {sx, sxy, (cuuint64_t)ll.pld * 4};
        const cuuint32_t box[4] = {T4W, TY + 2, 1, 1};
        make_map(&tp, ll.pbase, 4, dims, strides, box);
    }
    {
        const cuuint64_t dims[3] = {(cuuint64_t)g.Nx, (cuuint64_t)g.Ny, (cuuint64_t)g.Nz};
        const cuuint64_t strides[2] = {sx, sxy};
        const cuuint32_t box[3] = {T4W, TY + 2, 1};
        make_map(&td, D, 3, dims, strides, box);
    }
    {
        const cuuint64_t dims[4] = {(cuuint64_t)g.Nx, (cuuint64_t)g.Ny, (cuuint64_t)g.Nz, (cuuint64_t)ll.gslots};
        const cuuint64_t strides[3] = {sx, sxy, (cuuint64_t)g.ld * 4};
        const cuuint32_t box[4] = {T4X, TY, 1, 1};
        make_map(&tg, ll.gbase, 4, dims, strides, box);
    }
    (void)sxyz;
    const size_t smem = s4t_smem<ZL, TY>();
    static int occ[64] = {};
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !occ[dev]) {
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_stencil4t<ZL, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int o = 0;
        RCG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_stencil4t<ZL, TY>, 16 * TY, smem));
        if (dev >= 0 && dev < 64) occ[dev] = std::max(o, 1);
    }
    const int o = (dev >= 0 && dev < 64) ? occ[dev] : 1;
    const long long T = (long long)(g.Nx / T4X) * ((g.Ny + TY - 1) / TY), G = (ll.na + ZL - 1) / ZL;
    const long long resident = (long long)o * device_sms(dev);
    long long nzc = (4 * resident + T * G - 1) / (T * G);
    nzc = std::max<long long>(1, std::min<long long>(nzc, std::max(1, g.Nz / 8)));
    const int zc = (int)((g.Nz + nzc - 1) / nzc);
    nzc = (g.Nz + zc - 1) / zc;
    if (G > 65535) throw Error{RCG_ERR_INVALID, "k_stencil4t: grid extent"};
    k_stencil4t<ZL, TY><<<dim3((unsigned)(T * nzc), (unsigned)G), 16 * TY, smem, st>>>(
        tp, td, tg, g, ll.gbase, diag, q, ll.alist, ll.na, active, dots, prof, zc);
}



// Stencil variants: 0 the row kernel k_stencil4 (any Nx % 4 == 0), 1 the
// plane-ring kernel k_stencil4z (3D, 256 % (Nx / 4) == 0), 2 + the
// z-marching kernel k_stencil4r<TX, ZL> for TX in {4, 8, 16, 32} (TX | Nx/4),
// ZL in {1, 2, 4}: id 2 + 3 log2(TX / 4) + log2(ZL), in the default grid
// order; and with registers for 3 CTAs per SM: 14 <16,2>, 15 <8,2>.
// (Chunked lane-group orders for many lanes measured no faster than the
// tile-first order at 64-256 lanes of the 192^3 grid: the kernel is not
// short of DRAM bandwidth there but of memory-level parallelism.)
constexpr int S4_TXS[4] = {4, 8, 16, 32};
constexpr int S4_ZLS[3] = {1, 2, 4};
constexpr int S4_NVAR = 2 + 12 + 2 + 3;   // + the TMA plane-ring kernel k_stencil4t <2,16>, <2,8>, <4,8>
static_assert(S4_NVAR == RCG_STENCIL_VARIANTS, "variant count");

bool s4_variant_ok(const Grid &g, int v) {
    if (v == 0) return cg4_supported(g);
    if (v == 1) return stencil4z_supported(g);
    if (v >= 16 && v < S4_NVAR) return s4t_supported(g);
    if (v < 2 || v >= S4_NVAR) return false;
    const int tx = v >= 14 ? (v == 15 ? 8 : 16) : S4_TXS[(v - 2) / 3];
    return cg4_supported(g) && g.Ny > 1 && (g.Nx / 4) % tx == 0 && g.n < (1LL << 31);
}

std::string s4_variant_name(int v) {
    if (v == 16) return "k_stencil4t<2,16> (TMA plane ring)";
    if (v == 17) return "k_stencil4t<2,8> (TMA plane ring)";
    if (v == 18) return "k_stencil4t<4,8> (TMA plane ring)";
    if (v == 0) return "k_stencil4 (rows)";
    if (v == 1) return "k_stencil4z (plane ring)";
    if (v >= 14) return std::string(v == 15 ? "k_stencil4r<8,2>" : "k_stencil4r<16,2>") + ", 3 CTAs per SM";
    return "k_stencil4r<" + std::to_string(S4_TXS[(v - 2) / 3]) + "," + std::to_string(S4_ZLS[(v - 2) % 3]) + ">";
}

void s4_launch(int v, cudaStream_t st, const Grid &g, const float *D, const float *const *diag, const float *const *p,
               float *const *q, const LaneList &ll, const int *active, double *dots, unsigned long long *prof) {
    const long long nv = g.n >> 2;
    switch (v) {
        case 0:
            k_stencil4<<<dim3(gx_for(nv, ll.na, 8), ll.na), kThreads, 0, st>>>(g, D, diag, p, q, ll.alist, active, dots,
                                                                             prof);
            break;
        case 1: launch_s4z(st, g, D, diag, p, q, ll, active, dots, prof); break;
#define RCG_S4R(ID, TX, ZLV) case ID: launch_s4r<TX, ZLV>(st, g, D, diag, p, q, ll, active, dots, prof); break;
        RCG_S4R(2, 4, 1) RCG_S4R(3, 4, 2) RCG_S4R(4, 4, 4)
        RCG_S4R(5, 8, 1) RCG_S4R(6, 8, 2) RCG_S4R(7, 8, 4)
        RCG_S4R(8, 16, 1) RCG_S4R(9, 16, 2) RCG_S4R(10, 16, 4)
        RCG_S4R(11, 32, 1) RCG_S4R(12, 32, 2) RCG_S4R(13, 32, 4)
#undef RCG_S4R
        case 14: launch_s4r<16, 2, 3>(st, g, D, diag, p, q, ll, active, dots, prof); break;
        case 15: launch_s4r<8, 2, 3>(st, g, D, diag, p, q, ll, active, dots, prof); break;
        case 16: launch_s4t<2, 16>(st, g, D, diag, q, ll, active, dots, prof); break;
        case 17: launch_s4t<2, 8>(st, g, D, diag, q, ll, active, dots, prof); break;
        case 18: launch_s4t<4, 8>(st, g, D, diag, q, ll, active, dots, prof); break;
        default: throw Error{RCG_ERR_INVALID, "unknown stencil variant"};
    }
    count_launch();
    RCG_CHECK_LAUNCH();
}

// The autotuner: the first float32 iteration of a (device, grid, lane-count
// class) times every variant that supports the grid on that iteration's own
// lanes (CUDA events, one warm-up and three timed launches each, p^T q into a
// scratch buffer) and keeps the fastest; later iterations look it up.
struct TuneKey {
    int dev, Nx, Ny, Nz, cls;
    bool operator<(const TuneKey &o) const {
        return std::tie(dev, Nx, Ny, Nz, cls) < std::tie(o.dev, o.Nx, o.Ny, o.Nz, o.cls);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;
std::vector<std::string> g_tune_log;

int lane_class(int na) {
    int c = 0;
    while ((1 << c) < na && c < 14) ++c;
    return c;
}

int s4_tuned(cudaStream_t st, const Grid &g, const float *D, const float *const *diag, const float *const *p,
             float *const *q, const LaneList &ll, const int *active, int mcap) {
    int dev = 0;
    RCG_CUDA_TRY(cudaGetDevice(&dev));
    const TuneKey key{dev, g.Nx, g.Ny, g.Nz, lane_class(ll.na)};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) return it->second;
    }
    double *scr = nullptr;
    RCG_CUDA_TRY(cudaMalloc(&scr, sizeof(double) * (size_t)std::max(mcap, 1)));   // p^T q of lanes < mcap
    cudaEvent_t e0, e1;
    RCG_CUDA_TRY(cudaEventCreate(&e0));
    RCG_CUDA_TRY(cudaEventCreate(&e1));
    int best = -1;
    float best_ms = 0.f;
    std::string log = "stencil " + std::to_string(g.Nx) + "x" + std::to_string(g.Ny) + "x" + std::to_string(g.Nz) +
                      ", lanes <= " + std::to_string(1 << key.cls) + ":";
    try {
        for (int v = 0; v < S4_NVAR; ++v) {
            if (!s4_variant_ok(g, v) || (v >= 16 && !s4t_usable(g, ll))) continue;
            s4_launch(v, st, g, D, diag, p, q, ll, active, scr, nullptr);
            RCG_CUDA_TRY(cudaEventRecord(e0, st));
            for (int rep = 0; rep < 3; ++rep) s4_launch(v, st, g, D, diag, p, q, ll, active, scr, nullptr);
            RCG_CUDA_TRY(cudaEventRecord(e1, st));
            RCG_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            RCG_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            ms /= 3.f;
            char b[96];
            std::snprintf(b, sizeof b, " %s %.1f us;", s4_variant_name(v).c_str(), 1e3 * ms);
            log += b;
            if (best < 0 || ms < best_ms) { best = v; best_ms = ms; }
        }
    } catch (...) {
        cudaEventDestroy(e0); cudaEventDestroy(e1); cudaFree(scr);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RCG_CUDA_TRY(cudaFree(scr));
    log += " -> " + s4_variant_name(best);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
    g_tune_log.push_back(log);
    return best;
}

}  // namespace

int stencil_take_error(cudaStream_t st) {
    int h = 0, z = 0;
    RCG_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, g_s4t_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    RCG_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) RCG_CUDA_TRY(cudaMemcpyToSymbolAsync(g_s4t_err, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st));
    if (h) RCG_CUDA_TRY(cudaStreamSynchronize(st));
    return h;
}

std::string stencil_tuning_report() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::string s;
    for (auto &l : g_tune_log) s += l + "\n";
    return s;
}

const char *stencil_variant_name(int v) {
    static std::string names[S4_NVAR];
    if (v < 0 || v >= S4_NVAR) return nullptr;
    static std::once_flag once;
    std::call_once(once, [] { for (int i = 0; i < S4_NVAR; ++i) names[i] = s4_variant_name(i); });
    return names[v].c_str();
}

int stencil_variant_ok(const Grid &g, int v) { return s4_variant_ok(g, v) ? 1 : 0; }

// q = A~_s p on ncols float32 columns with stencil variant v (-1: the tuned
// choice), p^T q added into dots[c] (device, ncols doubles): a parity and
// timing entry for the kernels of the inner iteration.
void stencil4_apply(cudaStream_t st, const Grid &g, const float *D, const float *const *diag, const float *const *p,
                    float *const *q, int ncols, const int *lanes, const int *active, double *dots, int v,
                    const float *pbase, long long pld, const float *gbase, int gslots) {
    LaneList ll{lanes, ncols, nullptr, nullptr, nullptr, 0};
    ll.pbase = pbase; ll.pld = pld; ll.pcols = ncols; ll.gbase = gbase; ll.gslots = gslots;
    if (v >= 16 && !s4t_usable(g, ll)) throw Error{RCG_ERR_INVALID, "the TMA stencil needs the columns' layout"};
    if (ncols <= 0) return;
    if (v < 0) v = s4_tuned(st, g, D, diag, p, q, ll, active, ncols);
    if (!s4_variant_ok(g, v)) throw Error{RCG_ERR_INVALID, "stencil variant does not support this grid"};
    s4_launch(v, st, g, D, diag, p, q, ll, active, dots, nullptr);
}

// One float32 iteration t over the active lanes (see the file comment).
void cg_iteration4(cudaStream_t st, const Grid &g, const float *D, const float *const *diag_of_col,
                   const float *const *p_ptr, float *const *q_ptr, LaneGeom gm, LaneState ls, LaneList ll, int t,
                   float *mu, float *beta, KTimer *kt) {
    if (ll.na <= 0) return;
    const int sprev = (t - 1) % 3, scur = t % 3, snext = (t + 1) % 3, spq = t % 2, sw = t % 2;
    const bool tm = kt && kt->on;
    // the tuner's launches (first iteration of a grid and lane class only) run
    // before the timed launch
    const int sv = s4_tuned(st, g, D, diag_of_col, p_ptr, q_ptr, ll, ls.active, ls.m);
    cudaEvent_t e = tm ? kt->start(st) : nullptr;
    s4_launch(sv, st, g, D, diag_of_col, p_ptr, q_ptr, ll, ls.active, ls.pq + (long long)spq * ls.m, ls.prof);
    if (tm) { kt->stop(0, e, st); e = kt->start(st); }
    // node range per CTA for the tile kernels: a multiple of SN, `slots` CTAs in total
    auto tile_chunk = [&](long long &z, long long slots = 6LL * 152) {
        z = std::max<long long>(1, slots / ll.ntiles);
        const long long maxz = (g.n + 4 * SN - 1) / (4 * SN);
        if (z > maxz) z = maxz;
        if (z < 1) z = 1;
        long long chunk = (g.n + z - 1) / z;
        chunk = (chunk + SN - 1) / SN * SN;
        z = (g.n + chunk - 1) / chunk;
        return chunk;
    };
    const int kut = gm.k_u <= 4 ? 4 : gm.k_u <= 8 ? 8 : gm.k_u <= 12 ? 12 : 16;
    const bool fused = gm.k_u > 0;
    if (fused) {
        // the update with the shared deflation dots (one read of r)
        long long z;
        const long long chunk = tile_chunk(z, 4LL * 152);
        dim3 grid((unsigned)z, ll.ntiles);
// up to four private columns: the staged kernel; more: the register version
#define RCG_UUS(K, P) launch_update_u0s<K, P>(st, grid, g.n, gm, ls, ll, t, sprev, scur, spq, sw, chunk)
#define RCG_UU(K, P) k_update_u0<K, P><<<grid, kUU, 0, st>>>(g.n, gm, ls, ll.tile_lane, ll.tile_si, ll.tile_cnt, \
                                                                  t, sprev, scur, spq, sw, chunk)
#define RCG_UUK(K) if (gm.kp_sel <= 1) RCG_UUS(K, 1); else if (gm.kp_sel <= 2) RCG_UUS(K, 2); \
                   else if (gm.kp_sel <= 4) RCG_UUS(K, 4); else RCG_UU(K, KP_MAX)
        switch (kut) { case 4: RCG_UUK(4); break; case 8: RCG_UUK(8); break; case 12: RCG_UUK(12); break;
                       default: RCG_UUK(16); }
#undef RCG_UUK
#undef RCG_UU
#undef RCG_UUS
    } else if (gm.kp_sel <= 1) launch_update4<1>(st, g.n, gm, ls, ll, t, sprev, scur, spq, sw);
    else if (gm.kp_sel <= 2) launch_update4<2>(st, g.n, gm, ls, ll, t, sprev, scur, spq, sw);
    else if (gm.kp_sel <= 4) launch_update4<4>(st, g.n, gm, ls, ll, t, sprev, scur, spq, sw);
    else launch_update4<KP_MAX>(st, g.n, gm, ls, ll, t, sprev, scur, spq, sw);
    count_launch();
    RCG_CHECK_LAUNCH();
    if (tm) { kt->stop(1, e, st); e = kt->start(st); }
    if (tm) { kt->stop(2, e, st); e = kt->start(st); }
    k_mu<<<ll.na, 32, 0, st>>>(ls, ll.alist, sprev, scur, snext, sw, mu, beta, 0);
    count_launch();
    RCG_CHECK_LAUNCH();
    if (tm) { kt->stop(3, e, st); e = kt->start(st); }
    {
        direction_launch(st, kut, g.n, gm, ls, ll, mu, beta, t);
        count_launch();
        RCG_CHECK_LAUNCH();
    }
    if (tm) kt->stop(4, e, st);
}

// (Re)start of the lanes of ll (float32, Nx % 4 == 0) at iteration number t;
// the same steps as cg_restart in cg.cu.  k_lane_zero has run for these lanes.
void cg_restart4(cudaStream_t st, const Grid &g, LaneGeom gm, LaneState ls, LaneList ll, int t, float *mu,
                 float *beta, int *drop) {
    if (ll.na <= 0) return;
    const int scur = t % 3, snext = (t + 1) % 3, sprev = (t + 2) % 3;
    const int sw = t % 2, sA = (t + 1) % 2;
    const long long nv = g.n >> 2;
    long long z = (6LL * 152 + ll.ntiles - 1) / ll.ntiles;
    const long long maxz = (g.n + 4 * SN - 1) / (4 * SN);
    if (z > maxz) z = maxz;
    if (z < 1) z = 1;
    long long chunk = (g.n + z - 1) / z;
    chunk = (chunk + SN - 1) / SN * SN;
    z = (g.n + chunk - 1) / chunk;
    const dim3 tgrid((unsigned)z, ll.ntiles), lgrid(gx_for(nv, ll.na, 8), ll.na);
    const int kut = gm.k_u <= 4 ? 4 : gm.k_u <= 8 ? 8 : gm.k_u <= 12 ? 12 : 16;
#define RCG_U0(K, W, SLOT) u0dots_attr<K>(); \
    k_u0dots<K><<<tgrid, kThreads, u0_smem<K>(), st>>>(g.n, gm, ls, ll.tile_lane, ll.tile_si, ll.tile_cnt, SLOT, chunk, W)
#define RCG_U0S(W, SLOT) switch (kut) { case 4: RCG_U0(4, W, SLOT); break; case 8: RCG_U0(8, W, SLOT); break; \
                                    case 12: RCG_U0(12, W, SLOT); break; default: RCG_U0(16, W, SLOT); }
    // z = W^T r -> wv[sA]
    if (gm.k_u > 0) { RCG_U0S(1, sA); count_launch(); RCG_CHECK_LAUNCH(); }
    k_private_dots4<<<lgrid, kThreads, 0, st>>>(g.n, gm, ls, ll.alist, 0, sA, 0, 0);
    count_launch();
    RCG_CHECK_LAUNCH();
    // mu0 = Ginv z; x = W mu0; r -= A W mu0
    k_mu_only<<<ll.na, 32, 0, st>>>(ls, ll.alist, sA, mu);
    count_launch();
    RCG_CHECK_LAUNCH();
#define RCG_PJ(K) k_project4<K><<<tgrid, kThreads, 0, st>>>(g.n, gm, ll.tile_lane, ll.tile_si, ll.tile_cnt, mu, chunk)
    switch (kut) { case 4: RCG_PJ(4); break; case 8: RCG_PJ(8); break; case 12: RCG_PJ(12); break; default: RCG_PJ(16); }
#undef RCG_PJ
    count_launch();
    RCG_CHECK_LAUNCH();
    // the learned column served the projection only (RCG_LEARN_START)
    drop_last_private(st, ls, const_cast<int *>(gm.kp), drop, ls.nl);
    // rr and (A W)^T r -> rr[scur], wv[sw]
    if (gm.k_u > 0) { RCG_U0S(0, sw); count_launch(); RCG_CHECK_LAUNCH(); }
#undef RCG_U0S
#undef RCG_U0
    k_private_dots4<<<lgrid, kThreads, 0, st>>>(g.n, gm, ls, ll.alist, 1, sw, 1, scur);
    count_launch();
    RCG_CHECK_LAUNCH();
    // decision, mu, beta = 0, slot zeroing (wv[sA] is zeroed as wv[1 - sw]); p = r - W mu
    k_mu<<<ll.na, 32, 0, st>>>(ls, ll.alist, sprev, scur, snext, sw, mu, beta, 1);
    count_launch();
    RCG_CHECK_LAUNCH();
    long long zc;
    (void)zc;
    // no x step is pending at a restart (x = W mu0 was just set): iteration
    // number -2 matches no stamp
    direction_launch(st, kut, g.n, gm, ls, ll, mu, beta, -2);
    count_launch();
    RCG_CHECK_LAUNCH();
}

}  // namespace rcg
