// batch_adjoint.cu -- batched adjoint: the gradients of a loss on u_T with
// respect to u_0 and the coefficients, for many independent 2D FP32 grids
// of uneven size, stencil and length, in persistent launches replayed as one
// CUDA graph.  (No counterpart in the paper; the adjoint follows from
// differentiating the time loop of Section 3.3, and every pass reuses the
// N.5D-blocked warp tile of the forward sweep.)
//
// For a grid with one-step operator S (interior), g_T = dL/du_T:
//     g_t = S^T g_{t+1}          (transposed stencil: offsets -o_k, zero halo)
//     dL/dc_k = sum_t sum_p g_{t+1}[p] u_t[p + o_k]
// Schedule of one grid, with block degree nb and M = ceil(T / nb) blocks:
//   F_p, p = 0..M-2:   forward pass of degree nb, C[p] -> C[p+1]
//                      (checkpoints; C[0] = u_0);
//   then for m = M-1 down to 0 (block m: steps t0 = m nb .. t0 + nb_m - 1):
//   R_m (nb_m >= 2):   forward pass of degree nb_m - 1 from C[m] that stores
//                      every level: U[s] = u_{t0+s}, s = 1..nb_m-1;
//   B_m:               transposed pass of degree nb_m from g_{t0+nb_m} to
//                      g_{t0}; as each level q = 0..nb_m-1 (g_{t0+nb_m-q})
//                      passes through the warp's registers, the products
//                      g_{t0+nb_m-q}[p] u_{t0+nb_m-1-q}[p + o_k] are added
//                      to the warp's per-coefficient sums (u from C[m] and
//                      U, read back through L1/L2), so no level of g is
//                      ever stored and no separate reduction pass runs.
// Work items are (grid, x tile, stream block, pass), pass-major; a warp
// takes the next item, waits (bounded) until the 3x3 neighbourhood of tiles
// has finished the grid's previous pass, runs it and publishes its counter
// (the batched forward's queue).  Every pass of a grid uses the tiling of
// degree nb, so consecutive passes have the same tiles whatever their
// degree.  Grids are processed in waves whose work memory (checkpoints,
// levels, one g buffer, per-tile partial sums) fits a budget; waves run one
// after another in the graph.
//
// Determinism: each warp sums its tile's products in FP32 in a fixed order,
// reduces the 32 lanes in FP64 with a fixed shuffle tree and adds the result
// to its tile's FP64 slot; the passes of a tile are ordered by the counters,
// and a final kernel sums the slots of a grid in tile order.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "an5d.h"
#include "an5d_internal.h"
#include "sweep2d.cuh"

namespace an5d {

constexpr int ADJB_WARPS = 4;
constexpr int ADJB_MAX_N = 25;
// block degree per class (star R1, star R2, box R1, box R2): the backward
// pass holds the transposed levels and the gradient sums in registers
__host__ __device__ constexpr int adjb_nb(int cls) { return (cls % 2 == 0) ? 4 : 2; }

struct AdjGrid {
    const float *u0;   // C[0] = the forward input (caller's)
    float *gout;       // dL/du_0 (caller's), zero halo
    float *ck;         // checkpoints C[1..M-1], gstride elements apart
    float *ul;         // recomputed levels U[1..nb-1]
    float *gx;         // the second g buffer (zero halo)
    double *part;      // per tile: N FP64 partial sums of dL/dc
    int64_t gstride;   // elements between consecutive work grids
    int total;         // padded elements
    int pitch, ny, nx, radius, cls, nb, M, T;
    int lead, stride, tiles_x, hsn, nsb, counter_base;
    float c[ADJB_MAX_N];   // coefficients (canonical order)
    float mc[ADJB_MAX_N];  // mirrored: mc[k] = c of offset -o_k
};

enum : int { ADJ_FWD = 0, ADJ_REC = 1, ADJ_BWD = 2 };

struct AdjItem {
    int g, xt, sb, pass, kind, m, deg;
};

// Canonical offset k of a 2D stencil (star: centre, then (dx=i), (dy=i) for
// i = -R..-1, 1..R; box: dy outer, dx inner).
template <int SHAPE, int R> __host__ __device__ constexpr int adj_dy(int k)
{
    if (SHAPE == SH_BOX) return k / (2 * R + 1) - R;
    if (k == 0) return 0;
    const int j = (k - 1) / 2, i = j < R ? j - R : j - R + 1;
    return (k - 1) % 2 == 1 ? i : 0;
}
template <int SHAPE, int R> __host__ __device__ constexpr int adj_dx(int k)
{
    if (SHAPE == SH_BOX) return k % (2 * R + 1) - R;
    if (k == 0) return 0;
    const int j = (k - 1) / 2, i = j < R ? j - R : j - R + 1;
    return (k - 1) % 2 == 0 ? i : 0;
}

// Row observer of the backward pass: level q of the transposed sweep is
// g_{t0+NB-q}; its product with u_{t0+NB-1-q} at the N offsets goes into the
// warp's per-coefficient sums, over the tile's stored cells only.
template <int SHAPE, int R, int NB> struct CorrHook {
    static constexpr bool active = true;
    static constexpr int N = NCoeff2<SHAPE, R>::value;
    const float *u[NB];  // u[s] = u_{t0+s}, padded
    int pitch, y0, y1;
    unsigned store_bits;
    int colc[CELLS_PER_LANE];  // the lane's columns clamped into the row: a lane
                               // of the tile's overlap reads a valid cell it
                               // does not use instead of one outside the array
    float acc[N];

    template <typename C, int V> __device__ __forceinline__ void row(int q, int j, const C (&g)[V])
    {
        if (j < y0 || j >= y1) return;  // the same row for the whole warp
        const float *us = u[NB - 1 - q];
        float gm[V];
#pragma unroll
        for (int v = 0; v < V; ++v) gm[v] = (store_bits >> v) & 1u ? g[v] : 0.f;
#pragma unroll
        for (int dy = -R; dy <= R; ++dy) {
            bool used = false, shifted = false;
#pragma unroll
            for (int k = 0; k < N; ++k)
                if (adj_dy<SHAPE, R>(k) == dy) {
                    used = true;
                    shifted |= adj_dx<SHAPE, R>(k) != 0;
                }
            if (!used) continue;
            const float *rp = us + (int64_t)(j + dy) * pitch;
            float w[V];
#pragma unroll
            for (int v = 0; v < V; ++v) w[v] = __ldg(rp + colc[v]);
            float L[R], Rt[R];
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                // a stored cell's x neighbours lie inside the tile: the lanes
                // at the tile's edges hold only overlap cells (masked)
                L[d - 1] = shifted ? __shfl_up_sync(FULL_MASK, w[V - d], 1) : 0.f;
                Rt[d - 1] = shifted ? __shfl_down_sync(FULL_MASK, w[d - 1], 1) : 0.f;
            }
#pragma unroll
            for (int k = 0; k < N; ++k) {
                if (adj_dy<SHAPE, R>(k) != dy) continue;
                const int dx = adj_dx<SHAPE, R>(k);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int s = v + dx;
                    const float x = s < 0 ? L[-s - 1] : (s >= V ? Rt[s - V] : w[s]);
                    acc[k] = __fmaf_rn(gm[v], x, acc[k]);
                }
            }
        }
    }
};

struct AdjCoeffs {
    float c[ADJB_MAX_N];
};

__device__ __forceinline__ void adj_inval_ring(unsigned char *ring, int D, int slot_bytes)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        uint64_t *bars = reinterpret_cast<uint64_t *>(ring + D * slot_bytes);
        for (int s = 0; s < D; ++s)
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bars[s])) : "memory");
    }
    __syncwarp();
}

// Forward pass of degree BT (checkpoints).
template <int SHAPE, int R, int BT>
__device__ __noinline__ bool adj_fwd_tile(const Tile2D tg, float *dst, int *status, unsigned char *ring,
                                          const float *gc)
{
    constexpr int N = NCoeff2<SHAPE, R>::value;
    AdjCoeffs cf;
#pragma unroll
    for (int k = 0; k < N; ++k) cf.c[k] = gc[k];
    const bool ok = sweep2d_tile<SHAPE, R, BT, float, MODE_PLAIN, false, decltype(cf.c), decltype(cf.c), false, true>(
        tg, nullptr, dst, status, ring, cf.c, cf.c);
    using G = Sweep2DGeom<float, BT, R>;
    adj_inval_ring(ring, G::D, G::SLOT_BYTES);
    return ok;
}

// Recompute pass of degree BT storing levels 1..BT-1 into lv[1..BT-1] and
// level BT into dst.
template <int SHAPE, int R, int BT>
__device__ __noinline__ bool adj_rec_tile(const Tile2D tg, float *dst, float *const *lv, int *status,
                                          unsigned char *ring, const float *gc)
{
    constexpr int N = NCoeff2<SHAPE, R>::value;
    AdjCoeffs cf;
#pragma unroll
    for (int k = 0; k < N; ++k) cf.c[k] = gc[k];
    const bool ok = sweep2d_tile<SHAPE, R, BT, float, MODE_PLAIN, false, decltype(cf.c), decltype(cf.c), true, true>(
        tg, nullptr, dst, status, ring, cf.c, cf.c, lv);
    using G = Sweep2DGeom<float, BT, R>;
    adj_inval_ring(ring, G::D, G::SLOT_BYTES);
    return ok;
}

// Backward pass of degree BT (transposed stencil) with the gradient sums;
// u[s] = u_{t0+s}.  Adds the warp's sums to part[0..N-1] (lane 0).
template <int SHAPE, int R, int BT>
__device__ __noinline__ bool adj_bwd_tile(const Tile2D tg, float *dst, const float *const *u, double *part,
                                          int *status, unsigned char *ring, const float *gmc)
{
    constexpr int N = NCoeff2<SHAPE, R>::value;
    constexpr int V = CELLS_PER_LANE;
    AdjCoeffs cf;
#pragma unroll
    for (int k = 0; k < N; ++k) cf.c[k] = gmc[k];
    CorrHook<SHAPE, R, BT> hook;
#pragma unroll
    for (int s = 0; s < BT; ++s) hook.u[s] = u[s];
    const int lane = threadIdx.x & 31;
    const int col0 = tg.x0 + lane * V;
    hook.pitch = tg.pitch;
    hook.y0 = tg.y0;
    hook.y1 = tg.y1;
    hook.store_bits = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int col = col0 + v;
        if (col >= tg.sc0 && col < tg.sc1) hook.store_bits |= 1u << v;
        hook.colc[v] = min(max(col, 0), tg.pitch - 1);
    }
#pragma unroll
    for (int k = 0; k < N; ++k) hook.acc[k] = 0.f;
    const bool ok =
        sweep2d_tile<SHAPE, R, BT, float, MODE_PLAIN, false, decltype(cf.c), decltype(cf.c), false, true, POST_NONE,
                     CELLS_PER_LANE, CorrHook<SHAPE, R, BT>>(tg, nullptr, dst, status, ring, cf.c, cf.c, nullptr, 0.f,
                                                             0ull, &hook);
    using G = Sweep2DGeom<float, BT, R>;
    adj_inval_ring(ring, G::D, G::SLOT_BYTES);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double v = (double)hook.acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL_MASK, v, o);
        if (lane == 0) part[k] += v;
    }
    return ok;
}

template <int SHAPE, int R> constexpr int adj_ring_bytes()
{
    return Sweep2DGeom<float, adjb_nb((SHAPE == SH_STAR ? 0 : 2) + R - 1), R>::WARP_BYTES;
}
constexpr int adj_cmax(int a, int b) { return a > b ? a : b; }
constexpr int ADJB_WARP_BYTES = adj_cmax(adj_cmax(adj_ring_bytes<SH_STAR, 1>(), adj_ring_bytes<SH_STAR, 2>()),
                                         adj_cmax(adj_ring_bytes<SH_BOX, 1>(), adj_ring_bytes<SH_BOX, 2>()));
constexpr int ADJB_SMEM = ADJB_WARPS * ADJB_WARP_BYTES + 128;

template <int SHAPE, int R>
__device__ __forceinline__ bool adj_dispatch(const AdjItem &w, const AdjGrid &g, const Tile2D &tg0, int *status,
                                             unsigned char *ring)
{
    constexpr int NB = adjb_nb((SHAPE == SH_STAR ? 0 : 2) + R - 1);
    const int64_t gs = g.gstride;
    Tile2D tg = tg0;
    if (w.kind == ADJ_FWD) {
        tg.src = w.m == 0 ? g.u0 : g.ck + (w.m - 1) * gs;
        return adj_fwd_tile<SHAPE, R, NB>(tg, g.ck + w.m * gs, status, ring, g.c);
    }
    const float *cm = w.m == 0 ? g.u0 : g.ck + (w.m - 1) * gs;  // C[m]
    if (w.kind == ADJ_REC) {
        tg.src = cm;
        float *lv[NB];
#pragma unroll
        for (int s = 0; s < NB; ++s) lv[s] = s == 0 ? nullptr : g.ul + (s - 1) * gs;  // U[s]
        float *dst = g.ul + (w.deg - 1) * gs;                                       // U[deg]
        if constexpr (NB >= 2) {
            if (w.deg == 1) return adj_rec_tile<SHAPE, R, 1>(tg, dst, lv, status, ring, g.c);
        }
        if constexpr (NB >= 3) {
            if (w.deg == 2) return adj_rec_tile<SHAPE, R, 2>(tg, dst, lv, status, ring, g.c);
        }
        if constexpr (NB >= 4) {
            if (w.deg == 3) return adj_rec_tile<SHAPE, R, 3>(tg, dst, lv, status, ring, g.c);
        }
        return false;
    }
    // backward: g buffers alternate so that block 0 writes gout; block M-1
    // reads the one it does not write (the initial g_T)
    float *out = (w.m % 2 == 0) ? g.gout : g.gx;
    const float *in = (w.m % 2 == 0) ? g.gx : g.gout;
    tg.src = in;
    const float *u[NB];
#pragma unroll
    for (int s = 0; s < NB; ++s) u[s] = s == 0 ? cm : g.ul + (s - 1) * gs;
    double *part = g.part + (int64_t)(w.sb * g.tiles_x + w.xt) * NCoeff2<SHAPE, R>::value;
    if (w.deg == 1) return adj_bwd_tile<SHAPE, R, 1>(tg, out, u, part, status, ring, g.mc);
    if constexpr (NB >= 2) {
        if (w.deg == 2) return adj_bwd_tile<SHAPE, R, 2>(tg, out, u, part, status, ring, g.mc);
    }
    if constexpr (NB >= 3) {
        if (w.deg == 3) return adj_bwd_tile<SHAPE, R, 3>(tg, out, u, part, status, ring, g.mc);
    }
    if constexpr (NB >= 4) {
        if (w.deg == 4) return adj_bwd_tile<SHAPE, R, 4>(tg, out, u, part, status, ring, g.mc);
    }
    return false;
}

__global__ void __launch_bounds__(ADJB_WARPS * 32)
    adj_batch_kernel(const AdjGrid *__restrict__ grids, const AdjItem *__restrict__ items, int n_items, int *queue,
                     int *counters, int *status, int *abort_flag)
{
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *const base = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char *const ring = base + warp * ADJB_WARP_BYTES;
    while (true) {
        int it = 0;
        if (lane == 0) it = atomicAdd(queue, 1);
        it = __shfl_sync(FULL_MASK, it, 0);
        if (it >= n_items) break;
        if (__shfl_sync(FULL_MASK, lane == 0 ? *(volatile int *)abort_flag : 0, 0)) break;
        const AdjItem w = items[it];
        const AdjGrid &g = grids[w.g];
        // wait until the 3x3 neighbourhood has completed pass w.pass - 1
        bool ok = true;
        if (w.pass > 0 && lane < 9) {
            const int xt = w.xt + lane % 3 - 1, sb = w.sb + lane / 3 - 1;
            if (xt >= 0 && xt < g.tiles_x && sb >= 0 && sb < g.nsb) {
                const int *c = counters + g.counter_base + sb * g.tiles_x + xt;
                if (ld_acquire(c) < w.pass) {
                    const uint64_t t0 = global_ns();
                    while (ld_acquire(c) < w.pass) {
                        if (global_ns() - t0 > WAIT_LIMIT_NS) {
                            ok = false;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
            }
        }
        if (!__all_sync(FULL_MASK, ok)) {
            if (lane == 0) {
                atomicOr(status, STATUS_TIMEOUT);
                atomicExch(abort_flag, 1);
            }
            break;
        }
        // the neighbours' stores (generic proxy) before this warp's bulk reads (async proxy)
        asm volatile("fence.proxy.async.global;" ::: "memory");
        Tile2D tg;
        tg.src = nullptr;
        tg.total = g.total;
        tg.pitch = g.pitch;
        tg.ny = g.ny;
        tg.nx = g.nx;
        tg.x0 = g.radius - g.lead + w.xt * g.stride;
        tg.sc0 = max(g.radius, tg.x0 + g.lead);
        tg.sc1 = min(g.nx + g.radius, tg.x0 + g.lead + g.stride);
        tg.y0 = g.radius + w.sb * g.hsn;
        tg.y1 = min(tg.y0 + g.hsn, g.ny + g.radius);
        tg.stall = 0;
        bool done;
        switch (g.cls) {
        case 0: done = adj_dispatch<SH_STAR, 1>(w, g, tg, status, ring); break;
        case 1: done = adj_dispatch<SH_STAR, 2>(w, g, tg, status, ring); break;
        case 2: done = adj_dispatch<SH_BOX, 1>(w, g, tg, status, ring); break;
        default: done = adj_dispatch<SH_BOX, 2>(w, g, tg, status, ring); break;
        }
        if (!__all_sync(FULL_MASK, done)) {
            if (lane == 0) atomicExch(abort_flag, 1);
            break;
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence();  // this warp's stores before the counter
            atomicAdd(counters + g.counter_base + w.sb * g.tiles_x + w.xt, 1);
        }
    }
}

// Per grid (blockIdx.y) and padded row (blockIdx.x * 8 + warp): the halo of
// u_0 into every checkpoint and level grid; the g buffer that the last block
// reads := g_T on the interior, the other := 0 (both zero on the halo).
__global__ void adj_prep_kernel(const AdjGrid *__restrict__ grids, const float *const *__restrict__ gT)
{
    const AdjGrid &g = grids[blockIdx.y];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 8 + warp;
    const int R = g.radius, nyp = g.ny + 2 * R, nxp = g.pitch;
    if (row >= nyp) return;
    const float *src = g.u0 + (size_t)row * nxp;
    const bool halo_row = row < R || row >= nyp - R;
    const int nck = g.M > 0 ? g.M - 1 : 0;  // checkpoints C[1..M-1]
    const int nk = nck + (g.nb - 1);        // then the levels U[1..nb-1]
    for (int b = 0; b < nk; ++b) {
        float *d = (b < nck ? g.ck + (int64_t)b * g.gstride : g.ul + (int64_t)(b - nck) * g.gstride) +
                   (size_t)row * nxp;
        if (halo_row) {
            for (int x = lane; x < nxp; x += 32) d[x] = src[x];
        } else if (lane < 2 * R) {
            const int x = lane < R ? lane : nxp - 2 * R + lane;
            d[x] = src[x];
        }
    }
    const bool init_out = g.M == 0 || ((g.M - 1) % 2 == 1);
    float *gi = init_out ? g.gout : g.gx;
    float *gz = init_out ? g.gx : g.gout;
    const float *t = gT[blockIdx.y] + (size_t)row * nxp;
    for (int x = lane; x < nxp; x += 32) {
        const bool in = !halo_row && x >= R && x < nxp - R;
        gi[(size_t)row * nxp + x] = in ? t[x] : 0.f;
        gz[(size_t)row * nxp + x] = 0.f;
    }
}

// dc[g * 25 + k] = sum over the grid's tiles (in tile order) of part.
__global__ void adj_final_kernel(const AdjGrid *__restrict__ grids, int n, double *dc)
{
    const int gi = blockIdx.x;
    if (gi >= n) return;
    const AdjGrid &g = grids[gi];
    const int N = g.cls == 0 ? 5 : (g.cls == 1 ? 9 : (g.cls == 2 ? 9 : 25));
    const int tiles = g.tiles_x * g.nsb;
    for (int k = threadIdx.x; k < ADJB_MAX_N; k += blockDim.x) {
        double s = 0.0;
        if (k < N)
            for (int t = 0; t < tiles; ++t) s += g.part[(int64_t)t * N + k];
        dc[(int64_t)gi * ADJB_MAX_N + k] = s;
    }
}

}  // namespace an5d

using namespace an5d;

// ---------------------------------------------------------------------------
// Host side.

namespace {

struct Wave {
    std::vector<int> grids;            // indices into the batch
    std::vector<AdjItem> items;
    size_t work_bytes = 0;             // partial sums, then checkpoints, levels, g buffer
    size_t part_bytes = 0;             // the partial sums (zeroed per run)
    int n_counters = 0;
    int maxrows = 0;
    AdjGrid *d_grids = nullptr;
    AdjItem *d_items = nullptr;
    int *d_counters = nullptr;         // tile counters, then queue, abort, status
    const float **d_gT = nullptr;      // per grid of the wave: g_T
    double *d_dc = nullptr;            // per grid of the wave: 25 doubles
};

int mirror_k(int shape, int R, int k)
{
    if (shape == AN5D_BOX) return (2 * R + 1) * (2 * R + 1) - 1 - k;
    if (k == 0) return 0;
    const int j = (k - 1) / 2, axis = (k - 1) % 2;
    return 1 + 2 * (2 * R - 1 - j) + axis;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

size_t part_bytes_of(const AdjGrid &g) { return align256((size_t)g.tiles_x * g.nsb * ADJB_MAX_N * sizeof(double)); }

}  // namespace

struct an5d_adjoint_batch {
    int n = 0;
    std::vector<an5d_grid_desc> descs;
    std::vector<std::vector<double>> coeffs;
    std::vector<AdjGrid> grids;       // host copies (pointers set per run)
    std::vector<Wave> waves;
    size_t budget = 0;
    size_t work_bytes = 0;            // the largest wave's
    void *work = nullptr;
    int ctas = 0;
    double *h_dc = nullptr;           // pinned: n * 25
    double *d_dc_all = nullptr;       // n * 25
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    std::vector<const void *> last_u0, last_gT;
    std::vector<void *> last_gu;
    double cell_updates = 0;
    int64_t total_items = 0;
};

static thread_local std::string g_adjb_err;

static int afail(int st, const std::string &m)
{
    g_adjb_err = m;
    return st;
}

extern "C" const char *an5d_adjoint_batch_last_error(void) { return g_adjb_err.c_str(); }

extern "C" an5d_adjoint_batch *an5d_adjoint_batch_create(int n, const an5d_grid_desc *descs, size_t budget_bytes)
{
    if (n < 1 || !descs) {
        afail(AN5D_ERR_INVALID_ARG, "n must be >= 1 and descs non-NULL");
        return nullptr;
    }
    for (int i = 0; i < n; ++i) {
        const an5d_grid_desc &d = descs[i];
        if ((d.shape != AN5D_STAR && d.shape != AN5D_BOX) || d.radius < 1 || d.radius > 2 || !d.coeffs ||
            d.ny < 1 || d.nx < 1 || d.T < 0 || (d.ny + 2 * d.radius) * (d.nx + 2 * d.radius) >= (1ll << 31)) {
            afail(AN5D_ERR_INVALID_ARG, "grid " + std::to_string(i) +
                                            ": shape star/box, radius 1-2, extents >= 1, T >= 0, "
                                            "fewer than 2^31 padded cells");
            return nullptr;
        }
    }
    an5d_adjoint_batch *ab = new an5d_adjoint_batch();
    ab->n = n;
    ab->budget = budget_bytes ? budget_bytes : ((size_t)48 << 30);
    ab->descs.assign(descs, descs + n);
    ab->coeffs.resize(n);
    ab->grids.resize(n);
    // geometry and work memory per grid
    std::vector<size_t> need(n);
    for (int i = 0; i < n; ++i) {
        const an5d_grid_desc &d = descs[i];
        const int nc = an5d_coeff_count(2, d.shape, d.radius);
        ab->coeffs[i].assign(d.coeffs, d.coeffs + nc);
        ab->descs[i].coeffs = ab->coeffs[i].data();
        AdjGrid &g = ab->grids[i];
        memset(&g, 0, sizeof(g));
        const int R = d.radius;
        g.radius = R;
        g.cls = (d.shape == AN5D_STAR ? 0 : 2) + (R - 1);
        g.ny = (int)d.ny;
        g.nx = (int)d.nx;
        g.pitch = (int)d.nx + 2 * R;
        g.total = g.pitch * (g.ny + 2 * R);
        g.T = (int)d.T;
        g.nb = adjb_nb(g.cls);
        g.M = (int)((d.T + g.nb - 1) / g.nb);
        g.lead = g.nb * R;
        g.stride = 32 * CELLS_PER_LANE - 2 * g.nb * R;
        g.tiles_x = (g.nx + g.stride - 1) / g.stride;
        g.nsb = std::max(1, (g.ny + 255) / 256);
        g.hsn = (g.ny + g.nsb - 1) / g.nsb;
        g.hsn = std::max(g.hsn, std::min(g.ny, g.nb * R));
        g.nsb = (g.ny + g.hsn - 1) / g.hsn;
        for (int k = 0; k < nc; ++k) {
            g.c[k] = (float)d.coeffs[k];
            g.mc[k] = (float)d.coeffs[mirror_k(d.shape, R, k)];
        }
        const size_t gb = align256((size_t)g.total * 4);
        g.gstride = (int64_t)(gb / 4);
        const int ngrids = std::max(g.M - 1, 0) + (g.nb - 1) + 1;
        need[i] = ngrids * gb + part_bytes_of(g);
        ab->cell_updates += (double)d.ny * d.nx * d.T;
    }
    // waves: grids in order, each wave's work memory within the budget (a
    // grid larger than the budget gets a wave of its own)
    Wave cur;
    for (int i = 0; i < n; ++i) {
        if (!cur.grids.empty() && cur.work_bytes + need[i] > ab->budget) {
            ab->waves.push_back(std::move(cur));
            cur = Wave();
        }
        cur.grids.push_back(i);
        cur.work_bytes += need[i];
        cur.part_bytes += part_bytes_of(ab->grids[i]);
    }
    ab->waves.push_back(std::move(cur));
    for (auto &w : ab->waves) ab->work_bytes = std::max(ab->work_bytes, w.work_bytes);
    // Items and counters per wave: pass-major, grouped by (kind, class,
    // degree) inside a pass so that warps running at the same time share
    // code.  An item depends only on items of the previous pass, enumerated
    // earlier, so the queue cannot deadlock.  (Ordering the passes by their
    // estimated earliest start instead -- a list schedule of the grids'
    // chains -- measured slower: it spreads the long chains of the largest
    // grids over the whole queue.)
    for (auto &w : ab->waves) {
        int counter = 0, maxp = 0;
        std::vector<std::vector<AdjItem>> passes(w.grids.size());
        for (size_t gi = 0; gi < w.grids.size(); ++gi) {
            AdjGrid &g = ab->grids[w.grids[gi]];
            g.counter_base = counter;
            counter += g.tiles_x * g.nsb;
            w.maxrows = std::max(w.maxrows, g.ny + 2 * g.radius);
            auto &pl = passes[gi];
            for (int p = 0; p + 1 < g.M; ++p) pl.push_back(AdjItem{(int)gi, 0, 0, 0, ADJ_FWD, p, g.nb});
            for (int m = g.M - 1; m >= 0; --m) {
                const int nbm = std::min(g.nb, g.T - m * g.nb);
                if (nbm >= 2) pl.push_back(AdjItem{(int)gi, 0, 0, 0, ADJ_REC, m, nbm - 1});
                pl.push_back(AdjItem{(int)gi, 0, 0, 0, ADJ_BWD, m, nbm});
            }
            maxp = std::max(maxp, (int)pl.size());
        }
        for (int p = 0; p < maxp; ++p)
            for (int kind = 0; kind < 3; ++kind)
                for (int cls = 0; cls < 4; ++cls)
                    for (int deg = 4; deg >= 1; --deg)
                        for (size_t gi = 0; gi < w.grids.size(); ++gi) {
                            const AdjGrid &g = ab->grids[w.grids[gi]];
                            if (p >= (int)passes[gi].size()) continue;
                            const AdjItem &a = passes[gi][p];
                            if (a.kind != kind || g.cls != cls || a.deg != deg) continue;
                            for (int sb = 0; sb < g.nsb; ++sb)
                                for (int xt = 0; xt < g.tiles_x; ++xt)
                                    w.items.push_back(AdjItem{(int)gi, xt, sb, p, a.kind, a.m, a.deg});
                        }
        w.n_counters = counter;
        ab->total_items += (int64_t)w.items.size();
    }
    // device resources
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(adj_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ADJB_SMEM);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_batch_kernel, ADJB_WARPS * 32, ADJB_SMEM);
    if (e == cudaSuccess) e = cudaMalloc(&ab->work, std::max<size_t>(ab->work_bytes, 256));
    if (e == cudaSuccess) e = cudaMalloc(&ab->d_dc_all, sizeof(double) * ADJB_MAX_N * n);
    if (e == cudaSuccess) e = cudaMallocHost(&ab->h_dc, sizeof(double) * ADJB_MAX_N * n);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ab->graph_stream, cudaStreamNonBlocking);
    for (auto &w : ab->waves) {
        if (e == cudaSuccess) e = cudaMalloc(&w.d_grids, sizeof(AdjGrid) * w.grids.size());
        if (e == cudaSuccess && !w.items.empty()) e = cudaMalloc(&w.d_items, sizeof(AdjItem) * w.items.size());
        if (e == cudaSuccess) e = cudaMalloc(&w.d_counters, sizeof(int) * (w.n_counters + 3));
        if (e == cudaSuccess) e = cudaMalloc(&w.d_gT, sizeof(float *) * w.grids.size());
        if (e == cudaSuccess && !w.items.empty())
            e = cudaMemcpy(w.d_items, w.items.data(), sizeof(AdjItem) * w.items.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        afail(e == cudaErrorMemoryAllocation ? AN5D_ERR_OOM : AN5D_ERR_CUDA,
              std::string("adjoint batch setup: ") + cudaGetErrorString(e));
        an5d_adjoint_batch_destroy(ab);
        return nullptr;
    }
    ab->ctas = std::max(1, per_sm) * sms;
    return ab;
}

extern "C" void an5d_adjoint_batch_destroy(an5d_adjoint_batch *ab)
{
    if (!ab) return;
    cudaDeviceSynchronize();
    if (ab->graph) cudaGraphExecDestroy(ab->graph);
    if (ab->graph_stream) cudaStreamDestroy(ab->graph_stream);
    for (auto &w : ab->waves) {
        cudaFree(w.d_grids);
        cudaFree(w.d_items);
        cudaFree(w.d_counters);
        cudaFree(w.d_gT);
    }
    cudaFree(ab->work);
    cudaFree(ab->d_dc_all);
    cudaFreeHost(ab->h_dc);
    delete ab;
}

extern "C" int an5d_adjoint_batch_info(const an5d_adjoint_batch *ab, an5d_adjoint_batch_info_t *info)
{
    if (!ab || !info) return AN5D_ERR_INVALID_ARG;
    info->grids = ab->n;
    info->waves = (int)ab->waves.size();
    info->ctas = ab->ctas;
    info->items = ab->total_items;
    info->cell_updates = ab->cell_updates;
    info->work_bytes = ab->work_bytes;
    for (int c = 0; c < 4; ++c) info->class_nb[c] = adjb_nb(c);
    return AN5D_OK;
}

extern "C" int an5d_adjoint_batch_run(an5d_adjoint_batch *ab, const void *const *u0s, const void *const *gTs,
                                      void *const *grad_u0s, double *grad_coeffs, void *stream)
{
    if (!ab || !u0s || !gTs || !grad_u0s || !grad_coeffs) return afail(AN5D_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    bool same = ab->last_u0.size() == (size_t)ab->n;
    for (int i = 0; i < ab->n && same; ++i)
        same = ab->last_u0[i] == u0s[i] && ab->last_gT[i] == gTs[i] && ab->last_gu[i] == grad_u0s[i];
    if (!same) {
        for (int i = 0; i < ab->n; ++i) {
            if (!u0s[i] || !gTs[i] || !grad_u0s[i] ||
                (((uintptr_t)u0s[i] | (uintptr_t)gTs[i] | (uintptr_t)grad_u0s[i]) & 15))
                return afail(AN5D_ERR_INVALID_ARG, "grid " + std::to_string(i) + ": NULL or misaligned buffer");
            const size_t bytes = (size_t)ab->grids[i].total * 4;
            const char *a = (const char *)grad_u0s[i];
            for (const void *o : {u0s[i], gTs[i]}) {
                const char *b = (const char *)o;
                if (a < b + bytes && b < a + bytes)
                    return afail(AN5D_ERR_ALIAS, "grid " + std::to_string(i) + ": grad_u0 overlaps an input");
            }
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) return afail(AN5D_ERR_CUDA, "sync");
        // per wave: the grid table with this call's buffers and the work memory
        int dc_base = 0;
        for (auto &w : ab->waves) {
            std::vector<AdjGrid> tab(w.grids.size());
            std::vector<const float *> gt(w.grids.size());
            char *pp = (char *)ab->work;                // partial sums of the wave
            char *p = (char *)ab->work + w.part_bytes;  // grid buffers
            for (size_t gi = 0; gi < w.grids.size(); ++gi) {
                const int i = w.grids[gi];
                AdjGrid g = ab->grids[i];
                const size_t gb = (size_t)g.gstride * 4;
                g.u0 = (const float *)u0s[i];
                g.gout = (float *)grad_u0s[i];
                g.ck = (float *)p;
                p += (size_t)std::max(g.M - 1, 0) * gb;
                g.ul = (float *)p;
                p += (size_t)(g.nb - 1) * gb;
                g.gx = (float *)p;
                p += gb;
                g.part = (double *)pp;
                pp += part_bytes_of(g);
                tab[gi] = g;
                gt[gi] = (const float *)gTs[i];
            }
            if (cudaMemcpy(w.d_grids, tab.data(), sizeof(AdjGrid) * tab.size(), cudaMemcpyHostToDevice) !=
                    cudaSuccess ||
                cudaMemcpy(w.d_gT, gt.data(), sizeof(float *) * gt.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                return afail(AN5D_ERR_CUDA, "grid table upload");
            w.d_dc = ab->d_dc_all + (size_t)dc_base * ADJB_MAX_N;
            dc_base += (int)w.grids.size();
        }
        if (ab->graph) {
            cudaGraphExecDestroy(ab->graph);
            ab->graph = nullptr;
        }
        // capture: per wave, reset, preparation, the persistent sweep, the
        // final sums; waves share the work memory and run in order
        cudaStream_t cs = ab->graph_stream;
        cudaGraph_t gph = nullptr;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return afail(AN5D_ERR_CUDA, "graph capture begin");
        for (auto &w : ab->waves) {
            int *queue = w.d_counters + w.n_counters;
            cudaMemsetAsync(w.d_counters, 0, sizeof(int) * (w.n_counters + 3), cs);
            cudaMemsetAsync(ab->work, 0, w.part_bytes, cs);  // the partial sums start at zero
            adj_prep_kernel<<<dim3((w.maxrows + 7) / 8, (unsigned)w.grids.size()), 256, 0, cs>>>(w.d_grids, w.d_gT);
            if (!w.items.empty())
                adj_batch_kernel<<<ab->ctas, ADJB_WARPS * 32, ADJB_SMEM, cs>>>(
                    w.d_grids, w.d_items, (int)w.items.size(), queue, w.d_counters, queue + 2, queue + 1);
            adj_final_kernel<<<(unsigned)w.grids.size(), 32, 0, cs>>>(w.d_grids, (int)w.grids.size(), w.d_dc);
        }
        cudaError_t e = cudaStreamEndCapture(cs, &gph);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ab->graph, gph, 0);
        if (gph) cudaGraphDestroy(gph);
        if (e != cudaSuccess) return afail(AN5D_ERR_CUDA, std::string("graph: ") + cudaGetErrorString(e));
        ab->last_u0.assign(u0s, u0s + ab->n);
        ab->last_gT.assign(gTs, gTs + ab->n);
        ab->last_gu.assign(grad_u0s, grad_u0s + ab->n);
    }
    cudaError_t e = cudaGraphLaunch(ab->graph, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ab->h_dc, ab->d_dc_all, sizeof(double) * ADJB_MAX_N * ab->n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return afail(AN5D_ERR_CUDA, std::string("adjoint batch run: ") + cudaGetErrorString(e));
    // waves hold the grids in order: the dc rows are the grids' in order
    memcpy(grad_coeffs, ab->h_dc, sizeof(double) * ADJB_MAX_N * ab->n);
    int h[3] = {0, 0, 0};
    for (auto &w : ab->waves) {
        int hw[3] = {0, 0, 0};
        if (cudaMemcpy(hw, w.d_counters + w.n_counters, sizeof(hw), cudaMemcpyDeviceToHost) != cudaSuccess)
            return afail(AN5D_ERR_CUDA, "status read");
        h[1] |= hw[1];
        h[2] |= hw[2];
    }
    if (h[2] & STATUS_TIMEOUT) return afail(AN5D_ERR_TIMEOUT, "a bounded device wait gave up");
    if (h[1]) return afail(AN5D_ERR_TIMEOUT, "the adjoint batch was aborted");
    return AN5D_OK;
}
