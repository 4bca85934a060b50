// sweep2d.cuh -- 1.5D-blocked, temporally blocked 2D stencil sweep (sm_103a).
//
// Method (AN5D, Section 3.1 and Fig. 1): the grid is tiled along x and
// streamed along y.  A tile advances bT time levels per pass: level 0 is the
// streamed input row, level t (1..bT) lags level t-1 by R rows, and only
// level bT's compute region (the tile minus bT*R cells per side) is stored.
// The valid region shrinks by R cells per level (overlapped tiling,
// Section 2.3).  The streaming axis may be cut into stream blocks of hsn
// output rows (Section 3.2, "Division of Streaming Dimension").
//
// GB300 mapping (this library's design, not the paper's V100 scheme):
//  * one warp owns one tile of 32 lanes x 4 consecutive x cells; warps never
//    synchronise with each other: in-plane (x) neighbours travel by warp
//    shuffles, so the paper's shared-memory neighbour exchange and its
//    double buffering (Section 3.2) are not needed;
//  * input rows are staged by TMA (cp.async.bulk.tensor, 1D map over the
//    padded array) into a per-warp shared-memory ring guarded by mbarriers,
//    issued by one lane PREFETCH_ROWS rows ahead of the consumer;
//  * each time level keeps its 2R+1 most recent rows (star) or 2R+1 partial
//    sums (box) in registers, in a fixed ring indexed by row mod (2R+1), so
//    no register is ever shifted (Section 3.2 "Register Allocation"); the
//    streaming loop is unrolled by 2R+1 to make every ring index static;
//  * box stencils use per-row partial sums (associative stencil
//    optimisation, Sections 2.3/3.1): an arriving row of level t-1 adds its
//    (2R+1) x-terms to the 2R+1 pending rows of level t, in the canonical
//    order (dy outer, dx inner), so the result equals the plain fma chain;
//  * Dirichlet halo: halo rows are copied level to level (never computed);
//    in the two x-edge tiles the halo columns are reset to their input
//    values after every level (Section 3.1 "overwrites data in these regions
//    with their original values").
#pragma once

#include "an5d_internal.h"
#include <type_traits>

#include "device_common.cuh"

namespace an5d {

template <int SHAPE, int R> struct NCoeff2 {
    static constexpr int value = SHAPE == SH_STAR ? 4 * R + 1 : (2 * R + 1) * (2 * R + 1);
};

template <typename C, int N> struct CoeffBlock {
    C c[N];
};

template <typename S, int N> struct Sweep2DArgs {
    S *dst;
    int *status;
    int pitch;        // padded row length nx + 2R (elements)
    int ny, nx;       // interior extents
    int tile_stride;  // output columns per tile: 32*V - 2*bT*R
    int tiles_x;
    int hsn;          // output rows per stream block
    int total_warps;  // tiles_x * stream blocks
    CoeffBlock<typename StorageTraits<S>::C, N> k;
};

template <typename S, int BT, int R> struct Sweep2DGeom {
    static constexpr int V = CELLS_PER_LANE;
    static constexpr int A = StorageTraits<S>::ALIGN_ELEMS;
    static constexpr int TILE = 32 * V;
    static constexpr int ROWBUF = TILE + A;  // TMA box: tile + alignment slack
    static constexpr int SLOT_BYTES = ((ROWBUF * (int)sizeof(S) + 127) / 128) * 128;
    // A row stays in the ring for bT*R iterations after it is consumed (the
    // edge tiles re-read halo columns from it); PREFETCH_ROWS more are in flight.
    static constexpr int D = BT * R + PREFETCH_ROWS + 1;
    // Every warp's ring starts on a 128-byte boundary (TMA destination).
    static constexpr int WARP_BYTES = ((D * SLOT_BYTES + D * 8 + 127) / 128) * 128;
    // + 128 bytes to align the dynamic shared-memory base by hand.
    static constexpr int CTA_BYTES = WARPS_PER_CTA * WARP_BYTES + 128;
    static_assert(TILE - 2 * BT * R >= 8, "tile too narrow for bT*R");
    static_assert(R <= V, "radius must not exceed cells per lane");
};

// Per-warp TMA row ring.
template <typename S, int D, int SLOT_BYTES, int ROWBUF> struct RowRing {
    unsigned char *base;
    uint64_t *bars;
    const CUtensorMap *map;
    int pitch, x0, first_row, nrows;
    int *status;

    __device__ __forceinline__ int slot(int row) const { return pmod(row - first_row, D); }
    __device__ __forceinline__ uint32_t parity(int row) const
    {
        return (uint32_t)(((row - first_row) / D) & 1);
    }
    // Called by one lane.
    __device__ __forceinline__ void issue(int row) const
    {
        constexpr int A = StorageTraits<S>::ALIGN_ELEMS;
        const int lin = row * pitch + x0;
        const int s = slot(row);
        fence_proxy_async();
        mbar_expect_tx(&bars[s], ROWBUF * (int)sizeof(S));
        tma_load_1d(base + s * SLOT_BYTES, map, lin - pmod(lin, A), &bars[s]);
    }
    __device__ __forceinline__ const S *row_ptr(int row) const
    {
        constexpr int A = StorageTraits<S>::ALIGN_ELEMS;
        return reinterpret_cast<const S *>(base + slot(row) * SLOT_BYTES) + pmod(row * pitch + x0, A);
    }
    __device__ __forceinline__ bool wait(int row) const
    {
        return mbar_wait_warp(&bars[slot(row)], parity(row), status);
    }
    // After a failed wait: wait (bounded) for every copy still in flight so
    // that none lands in shared memory after the warp has exited.
    __device__ __forceinline__ void drain(int row) const
    {
        for (int r = row; r < row + PREFETCH_ROWS && r < nrows; ++r)
            if (!mbar_wait_warp(&bars[slot(r)], parity(r), status)) break;
    }
};

template <int SHAPE, int R, int BT, typename S, int MODE>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32)
    sweep2d_kernel(const __grid_constant__ CUtensorMap tmap,
                   const Sweep2DArgs<S, NCoeff2<SHAPE, R>::value> a)
{
    using C = typename StorageTraits<S>::C;
    using G = Sweep2DGeom<S, BT, R>;
    constexpr int V = G::V;
    constexpr int P = 2 * R + 1;
    constexpr int D = G::D;
    extern __shared__ __align__(128) unsigned char smem[];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * WARPS_PER_CTA + warp;
    if (gw >= a.total_warps) return;

    // ---- tile geometry (Section 3.1) ----
    const int xt = gw % a.tiles_x;
    const int sbk = gw / a.tiles_x;
    const int x0 = R - BT * R + xt * a.tile_stride;  // padded column of the tile's first cell
    const int nrows = a.ny + 2 * R;
    const int y0 = R + sbk * a.hsn;                 // output rows [y0, y1)
    const int y1 = min(y0 + a.hsn, a.ny + R);
    const int ys = max(0, y0 - BT * R);             // first input row needed
    const int ib0 = ys - ys % P;                    // streaming starts on a ring-period boundary
    const int iend = y1 + BT * R;                   // level bT emits row y1-1 at i = y1-1+bT*R

    const int col0 = x0 + lane * V;
    const int sc0 = max(R, x0 + BT * R);
    const int sc1 = min(a.nx + R, x0 + BT * R + a.tile_stride);
    unsigned halo_bits = 0, store_bits = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int col = col0 + v;
        if (col < R || col >= a.nx + R) halo_bits |= 1u << v;
        if (col >= sc0 && col < sc1) store_bits |= 1u << v;
    }
    const bool edge = __any_sync(FULL_MASK, halo_bits != 0);

    RowRing<S, D, G::SLOT_BYTES, G::ROWBUF> rs;
    unsigned char *const smem_al = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem) + 127) & ~uintptr_t(127));
    rs.base = smem_al + warp * G::WARP_BYTES;
    rs.bars = reinterpret_cast<uint64_t *>(rs.base + D * G::SLOT_BYTES);
    rs.map = &tmap;
    rs.pitch = a.pitch;
    rs.x0 = x0;
    rs.first_row = ib0;
    rs.nrows = nrows;
    rs.status = a.status;

    if (lane == 0) {
        for (int s = 0; s < D; ++s) mbar_init(&rs.bars[s], 1);
        fence_mbar_init();
        for (int r = ib0; r < ib0 + PREFETCH_ROWS && r < nrows; ++r) rs.issue(r);
    }
    __syncwarp();

    const auto &cf = a.k.c;
    S *const dst = a.dst;
    const int pitch = a.pitch;
    const int ny = a.ny;

    // Level-0 row i -> registers; prefetch row i + PREFETCH_ROWS.
    auto load_row = [&](int i, bool have, C (&row)[V]) -> bool {
        if (have) {
            if (!rs.wait(i)) {
                rs.drain(i);
                return false;
            }
            const S *src = rs.row_ptr(i) + lane * V;
#pragma unroll
            for (int v = 0; v < V; ++v) row[v] = load_c<S>(src[v]);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) row[v] = C(0);
        }
        __syncwarp();
        if (lane == 0 && i + PREFETCH_ROWS < nrows) rs.issue(i + PREFETCH_ROWS);
        return true;
    };

    auto store_row = [&](int j, const C (&res)[V]) {
        S *out = dst + (j * pitch + col0);
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (store_bits & (1u << v)) out[v] = to_storage<S>(res[v]);
    };

    // x-neighbours of a row held as V values per lane: L[d-1] = cell -d,
    // Rt[d-1] = cell V-1+d (relative to the lane's first cell).
    auto exchange = [&](const C (&row)[V], C (&L)[R], C (&Rt)[R]) {
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            L[d - 1] = __shfl_up_sync(FULL_MASK, row[V - d], 1);
            Rt[d - 1] = __shfl_down_sync(FULL_MASK, row[d - 1], 1);
        }
    };

    if constexpr (SHAPE == SH_STAR) {
        // ring[t][r % P] = level-t row r, t = 0..bT-1
        C ring[BT][P][V];
#pragma unroll
        for (int t = 0; t < BT; ++t)
#pragma unroll
            for (int s = 0; s < P; ++s)
#pragma unroll
                for (int v = 0; v < V; ++v) ring[t][s][v] = C(0);

        auto group = [&](auto check_tag, int ib) -> bool {
            constexpr bool CHECK = decltype(check_tag)::value;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int i = ib + k;
                if (CHECK && i >= iend) return true;
                if (!load_row(i, !CHECK || i < nrows, ring[0][k])) return false;
#pragma unroll
                for (int t = 1; t <= BT; ++t) {
                    const int j = i - t * R;  // level-t row completed now
                    const int sj = ((k - t * R) % P + P) % P;
                    if (CHECK && (j < R || j >= ny + R)) {  // halo row: fixed value
                        if (t < BT) {
#pragma unroll
                            for (int v = 0; v < V; ++v) ring[t][sj][v] = ring[t - 1][sj][v];
                        }
                        continue;
                    }
                    if (t == BT && (j < y0 || j >= y1)) continue;
                    C L[R], Rt[R];
                    exchange(ring[t - 1][sj], L, Rt);
                    Acc<MODE, C> acc[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[v].first(cf[0], ring[t - 1][sj][v]);
                    int kk = 1;
#pragma unroll
                    for (int ii = -R; ii <= R; ++ii) {
                        if (ii == 0) continue;
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const int s = v + ii;
                            const C xv = s < 0 ? L[-s - 1] : (s >= V ? Rt[s - V] : ring[t - 1][sj][s]);
                            acc[v].add(cf[kk], xv);
                        }
                        const int sy = ((k - t * R + ii) % P + P) % P;
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v].add(cf[kk + 1], ring[t - 1][sy][v]);
                        kk += 2;
                    }
                    C res[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) res[v] = level_round<S>(acc[v].result());
                    if (t < BT) {
                        if (edge) {
#pragma unroll
                            for (int v = 0; v < V; ++v)
                                if (halo_bits & (1u << v)) res[v] = ring[t - 1][sj][v];
                        }
#pragma unroll
                        for (int v = 0; v < V; ++v) ring[t][sj][v] = res[v];
                    } else {
                        store_row(j, res);
                    }
                }
            }
            return true;
        };

        for (int ib = ib0; ib < iend; ib += P) {
            const bool fast = (ib - BT * R >= R) && (ib + P - 1 - R < ny + R) && (ib + P <= iend);
            const bool ok = fast ? group(std::integral_constant<bool, false>{}, ib)
                                 : group(std::integral_constant<bool, true>{}, ib);
            if (!ok) return;
        }
    } else {
        // acc[t-1][r % P] = pending partial sum of level-t row r, t = 1..bT
        Acc<MODE, C> acc[BT][P][V];
#pragma unroll
        for (int t = 0; t < BT; ++t)
#pragma unroll
            for (int s = 0; s < P; ++s)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[t][s][v].set(C(0));

        auto group = [&](auto check_tag, int ib) -> bool {
            constexpr bool CHECK = decltype(check_tag)::value;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int i = ib + k;
                if (CHECK && i >= iend) return true;
                C in_row[V];
                if (!load_row(i, !CHECK || i < nrows, in_row)) return false;
#pragma unroll
                for (int t = 1; t <= BT; ++t) {
                    const int ar = i - (t - 1) * R;  // arriving level-(t-1) row
                    C L[R], Rt[R];
                    exchange(in_row, L, Rt);
#pragma unroll
                    for (int dy = -R; dy <= R; ++dy) {
                        const int b = ar - dy;  // pending level-t row receiving its dy term
                        const int sb = ((k - (t - 1) * R - dy) % P + P) % P;
                        if (CHECK && (b < R || b >= ny + R)) {
                            if (dy == 0 && t < BT) {
#pragma unroll
                                for (int v = 0; v < V; ++v) acc[t - 1][sb][v].set(in_row[v]);
                            }
                            continue;
                        }
#pragma unroll
                        for (int dx = -R; dx <= R; ++dx) {
                            const int kk = (dy + R) * P + (dx + R);
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                const int s = v + dx;
                                const C xv = s < 0 ? L[-s - 1] : (s >= V ? Rt[s - V] : in_row[s]);
                                if (dy == -R && dx == -R)
                                    acc[t - 1][sb][v].first(cf[kk], xv);
                                else
                                    acc[t - 1][sb][v].add(cf[kk], xv);
                            }
                        }
                    }
                    const int e = i - t * R;  // level-t row completed now
                    const int se = ((k - t * R) % P + P) % P;
                    C out_row[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) out_row[v] = level_round<S>(acc[t - 1][se][v].result());
                    if (t < BT) {
                        if (edge) {
                            const S *orig = rs.row_ptr(e) + lane * V;
#pragma unroll
                            for (int v = 0; v < V; ++v)
                                if (halo_bits & (1u << v)) out_row[v] = load_c<S>(orig[v]);
                        }
#pragma unroll
                        for (int v = 0; v < V; ++v) in_row[v] = out_row[v];
                    } else if (e >= y0 && e < y1) {
                        store_row(e, out_row);
                    }
                }
            }
            return true;
        };

        for (int ib = ib0; ib < iend; ib += P) {
            const bool fast = (ib - BT * R >= R) && (ib + P - 1 + R < ny + R) && (ib + P <= iend);
            const bool ok = fast ? group(std::integral_constant<bool, false>{}, ib)
                                 : group(std::integral_constant<bool, true>{}, ib);
            if (!ok) return;
        }
    }
}

// Host-side launcher of one instantiation.
template <int SHAPE, int R, int BT, typename S, int MODE>
cudaError_t launch_sweep2d(const PassDesc &d, cudaStream_t st)
{
    constexpr int N = NCoeff2<SHAPE, R>::value;
    using C = typename StorageTraits<S>::C;
    using G = Sweep2DGeom<S, BT, R>;
    Sweep2DArgs<S, N> a;
    a.dst = static_cast<S *>(d.dst);
    a.status = d.status;
    a.pitch = static_cast<int>(d.pitch);
    a.ny = d.ny;
    a.nx = d.nx;
    a.tile_stride = d.tile_stride_x;
    a.tiles_x = d.tiles_x;
    a.hsn = d.hsn;
    a.total_warps = d.total_units;
    for (int k = 0; k < N; ++k) a.k.c[k] = static_cast<C>(d.coeffs[k]);
    auto fn = sweep2d_kernel<SHAPE, R, BT, S, MODE>;
    if (G::CTA_BYTES > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             G::CTA_BYTES);
        if (e != cudaSuccess) return e;
    }
    fn<<<d.ctas, WARPS_PER_CTA * 32, G::CTA_BYTES, st>>>(d.tmap, a);
    return cudaGetLastError();
}

template <int SHAPE, int R, int BT, typename S, int MODE>
KernelEntry entry2d(int dtype)
{
    using G = Sweep2DGeom<S, BT, R>;
    KernelEntry e;
    e.key = KernelKey{2, SHAPE, R, dtype, BT};
    e.launch = &launch_sweep2d<SHAPE, R, BT, S, MODE>;
    e.func = reinterpret_cast<const void *>(&sweep2d_kernel<SHAPE, R, BT, S, MODE>);
    e.threads = WARPS_PER_CTA * 32;
    e.smem_bytes = G::CTA_BYTES;
    e.tile_x = G::TILE;
    e.tile_y = 1;
    e.units_per_cta = WARPS_PER_CTA;
    return e;
}

}  // namespace an5d
