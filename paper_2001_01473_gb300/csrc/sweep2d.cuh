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
//  * one warp owns one tile of 32 lanes x V consecutive x cells (V = 4; a
//    variant with V = 6 loses a smaller share of its tile to the overlap
//    at the degrees that fit the same registers); warps never
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
#include <cstring>
#include <type_traits>

#include "device_common.cuh"

namespace an5d {

template <int SHAPE, int R> struct NCoeff2 {
    static constexpr int value = SHAPE == SH_STAR ? 4 * R + 1 : (2 * R + 1) * (2 * R + 1);
};

template <typename S, int N> struct Sweep2DArgs {
    S *dst;
    int *status;
    int pitch;        // padded row length nx + 2R (elements)
    int ny, nx;       // interior extents
    int tile_stride;  // output columns per tile: 32*V - 2*bT*R
    int xb0;          // padded column where tile 0's compute region starts
    int tiles_x;
    int hsn;          // output rows per stream block
    int total_warps;  // tiles_x * stream blocks
    int stall_test;   // fault injection (tests only): warp 0's first row never completes
    CoeffBlock<typename StorageTraits<S>::C, N> k;
    CoeffBlock<unsigned long long, N> kp;  // FP32: (c_k, c_k) packed pairs for f32x2 arithmetic
    typename StorageTraits<S>::C post_c;   // divisor or reciprocal (division-type stencils)
    unsigned long long post_p;             // FP32: (post_c, post_c)
};

// One 8-byte pair of FP32 cells to global memory, stored if bit `bit` of
// `mask` is set.
__device__ __forceinline__ void st_pair_pred(float *p, float a, float b, unsigned mask, int bit)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q st.global.v2.f32 [%0], {%1, %2};\n\t}" ::"l"(p),
                 "f"(a), "f"(b), "r"(mask & (1u << bit))
                 : "memory");
}

template <typename S, int BT, int R, int V_ = CELLS_PER_LANE> struct Sweep2DGeom {
    static constexpr int V = V_;  // consecutive x cells per lane
    static constexpr int P = 2 * R + 1;  // register-ring period = unroll factor
    static constexpr int A = StorageTraits<S>::ALIGN_ELEMS;
    static constexpr int TILE = 32 * V;
    static constexpr int ROWBUF = TILE + A;  // TMA box: tile + alignment slack
    static constexpr int SLOT_BYTES = ((ROWBUF * (int)sizeof(S) + 127) / 128) * 128;
    // Rows are requested PF rows ahead (a multiple of P, at least PREFETCH_ROWS).
    static constexpr int PF = ((PREFETCH_ROWS + P - 1) / P) * P;
    // A row stays in the ring bT*R iterations after it was consumed (edge
    // tiles re-read their halo columns from it) while the next PF + P rows
    // are in flight; the depth is a multiple of P so that a group of P rows
    // occupies P consecutive slots of one mbarrier phase.
    static constexpr int D = ((PF + P + BT * R + P - 1) / P) * P;
    // Every warp's ring starts on a 128-byte boundary (TMA destination).
    static constexpr int WARP_BYTES = ((D * SLOT_BYTES + D * 8 + 127) / 128) * 128;
    // + 128 bytes to align the dynamic shared-memory base by hand.
    static constexpr int CTA_BYTES = WARPS_PER_CTA * WARP_BYTES + 128;
    static_assert(TILE - 2 * BT * R >= 8, "tile too narrow for bT*R");
    static_assert(R <= V, "radius must not exceed cells per lane");
    static_assert(PF <= 32, "prefetch lanes");
    static_assert(ROWBUF <= 256, "one TMA box holds at most 256 elements per dimension");
};

// CTAs per SM the register budget is sized for: the level rings need
// bT * (2R+1) * V values per thread, plus registers for addressing,
// accumulators and shuffled neighbours.
// Box stencils keep the arriving row and its shifted copies live as well.
template <typename S, int SHAPE, int BT, int R, int MODE, int V_ = CELLS_PER_LANE>
struct Sweep2DOccupancy {
    static constexpr int words =
        (int)(sizeof(typename StorageTraits<S>::C) / 4) * (MODE == MODE_DOT2 ? 2 : 1);
    static constexpr int regs = BT * (2 * R + 1) * V_ * words +
                                (SHAPE == SH_STAR ? 34 + 10 * R + 20 * (words - 1)
                                                    : 40 + 2 * (2 * R + 1) * (2 * R + 1) + 8 * R * words);
    static constexpr int raw = 65536 / (WARPS_PER_CTA * 32 * (((regs + 7) / 8) * 8));
    static constexpr int value = raw < 1 ? 1 : (raw > 8 ? 8 : raw);
};

// Geometry of one warp tile of one pass.
struct Tile2D {
    const void *src;  // source array (RAW row copies only)
    int total;        // elements of the source array (RAW row copies only)
    int pitch;     // padded row length nx + 2R (elements)
    int ny, nx;    // interior extents
    int x0;        // padded column of the tile's first cell
    int sc0, sc1;  // columns stored by this tile: [sc0, sc1)
    int y0, y1;    // rows stored by this tile (its stream block): [y0, y1)
    int stall;     // fault injection (tests only): the first row's wait cannot complete
};

// Default row observer of sweep2d_tile: none.  A row observer sees every
// interior row of levels 0..BT-1 as it is produced (level 0: the staged input
// row), with the warp's V cells per lane; the adjoint's coefficient gradient
// accumulates its products there.  Called by all 32 lanes.
struct NoRowHook {
    static constexpr bool active = false;
    template <typename C, int V> __device__ __forceinline__ void row(int, int, const C (&)[V]) {}
};

// One warp advances one tile of one stream block by BT time levels: it
// streams the source rows through its TMA ring and level registers and
// stores the level-BT rows [y0, y1) x [sc0, sc1).  The caller owns the
// warp's shared-memory ring (Sweep2DGeom::WARP_BYTES, 128-byte aligned).
// cf[k] are the coefficients, cp[k] the same as packed (c_k, c_k) pairs
// (used when PACK).  With LEVELS (scalar paths only) the intermediate levels
// t = 1..BT-1 are stored as well, level t into lvl[t], over the same region.
// With RAW the rows are fetched by non-tensor bulk copies from tg.src
// (clamped to the array; the array's last partial 16-byte chunk by plain
// loads) instead of through the tensor map: no descriptor to fetch, for
// callers that switch arrays often.  HOOK (scalar paths) observes the interior
// rows of levels 0..BT-1 (NoRowHook: none).  With POST (division-type stencils) every
// level's weighted sum is divided by post_c, or multiplied by it when post_c
// is the reciprocal (post_p: the pair (post_c, post_c)).  Returns false if a
// bounded wait gave up.
template <int SHAPE, int R, int BT, typename S, int MODE, bool PACK, typename CF, typename CP,
          bool LEVELS = false, bool RAW = false, int POST = POST_NONE, int V_ = CELLS_PER_LANE,
          typename HOOK = NoRowHook>
__device__ __forceinline__ bool sweep2d_tile(const Tile2D tg, const CUtensorMap *tmap, S *const dst,
                                             int *const status, unsigned char *const ring,
                                             const CF &cf, const CP &cp, S *const *lvl = nullptr,
                                             const typename StorageTraits<S>::C post_c = 0,
                                             const f2_t post_p = 0, HOOK *hook = nullptr)
{
    using C = typename StorageTraits<S>::C;
    using G = Sweep2DGeom<S, BT, R, V_>;
    constexpr int V = G::V;
    constexpr int P = G::P;
    constexpr int D = G::D;
    constexpr int A = G::A;
    constexpr int PF = G::PF;

    const int lane = threadIdx.x & 31;
    const int x0 = tg.x0;
    const int ny = tg.ny;
    const int pitch = tg.pitch;
    const int nrows = ny + 2 * R;
    const int y0 = tg.y0, y1 = tg.y1;
    const int ys = max(0, y0 - BT * R);             // first input row needed
    const int ib0 = ys - ys % P;                    // streaming starts on a ring-period boundary
    const int iend = y1 + BT * R;                   // level bT emits row y1-1 at i = y1-1+bT*R
    const int rend = min(nrows, iend);              // rows requested: exactly the rows consumed

    const int col0 = x0 + lane * V;
    unsigned halo_bits = 0, store_bits = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int col = col0 + v;
        if (col < R || col >= tg.nx + R) halo_bits |= 1u << v;
        if (col >= tg.sc0 && col < tg.sc1) store_bits |= 1u << v;
    }
    const bool edge = __any_sync(FULL_MASK, halo_bits != 0);
    uint64_t *const bars = reinterpret_cast<uint64_t *>(ring + D * G::SLOT_BYTES);

    // TMA of padded row r into ring slot s (one lane).  The copy starts at the
    // 16-byte boundary at or below the tile's first cell of that row.
    auto issue = [&](int r, int s) {
        const int lin = r * pitch + x0;
        fence_proxy_async();
        if constexpr (!RAW) {
            mbar_expect_tx(&bars[s], G::ROWBUF * (int)sizeof(S));
            tma_load_1d(ring + s * G::SLOT_BYTES, tmap, lin & ~(A - 1), &bars[s]);
        } else {
            const int a0 = lin & ~(A - 1);             // window [a0, a0 + ROWBUF)
            const int whole = tg.total & ~(A - 1);     // 16-byte chunks of the array
            const int lo = max(a0, 0), hi = min(a0 + G::ROWBUF, whole);
            S *slot = reinterpret_cast<S *>(ring + s * G::SLOT_BYTES);
            const S *srcp = static_cast<const S *>(tg.src);
            for (int e = max(lo, whole); e < min(a0 + G::ROWBUF, tg.total); ++e) slot[e - a0] = srcp[e];
            if (hi > lo) {
                mbar_expect_tx(&bars[s], (hi - lo) * (int)sizeof(S));
                bulk_load(slot + (lo - a0), srcp + lo, (hi - lo) * (int)sizeof(S), &bars[s]);
            } else {
                mbar_expect_tx(&bars[s], 0);
            }
        }
    };
    auto row_in_slot = [&](int r, int s) -> const S * {
        return reinterpret_cast<const S *>(ring + s * G::SLOT_BYTES) + ((r * pitch + x0) & (A - 1)) +
               lane * V;
    };

    if (lane == 0) {
        for (int s = 0; s < D; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (tg.stall && lane == 0 && ib0 < rend) mbar_expect_tx_only(&bars[0], 16);  // never delivered
    __syncwarp();
    if (lane < PF && ib0 + lane < rend) issue(ib0 + lane, lane);  // rows ib0 .. ib0+PF-1

    // Ring position of the group that starts at row ib: slots sb .. sb+P-1,
    // all in mbarrier phase `par`.
    int sb = 0;
    uint32_t par = 0;

    auto exchange = [&](const C (&row)[V], C (&L)[R], C (&Rt)[R]) {
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            L[d - 1] = __shfl_up_sync(FULL_MASK, row[V - d], 1);
            Rt[d - 1] = __shfl_down_sync(FULL_MASK, row[d - 1], 1);
        }
    };
    auto store_row_to = [&](S *base, int j, const C (&res)[V]) {
        S *out = base + (j * pitch + col0);
#pragma unroll
        for (int v = 0; v < V; ++v) st_pred<S>(out + v, to_storage<S>(res[v]), store_bits, v);
    };
    auto store_row = [&](int j, const C (&res)[V]) {
        S *out = dst + (j * pitch + col0);
#pragma unroll
        for (int v = 0; v < V; ++v) st_pred<S>(out + v, to_storage<S>(res[v]), store_bits, v);
    };
    // 8-byte pairs: with an even tile origin and an even pitch every row's
    // cells of a lane start on an 8-byte boundary, in the staging ring and in
    // the destination.  If no lane stores just one cell of a pair (interior
    // tiles at an even bT*R), the interior groups read and store pairs.
    constexpr bool PAIRABLE = std::is_same<S, float>::value && V % 2 == 0 && !RAW && !LEVELS;
    unsigned pair_bits = 0;  // bit h: cells 2h and 2h+1 are stored
    bool paired = false;
    if constexpr (PAIRABLE) {
        bool partial = false;
#pragma unroll
        for (int h = 0; h < V / 2; ++h) {
            const unsigned two = (store_bits >> (2 * h)) & 3u;
            if (two == 3u) pair_bits |= 1u << h;
            partial |= (two == 1u || two == 2u);
        }
        paired = __all_sync(FULL_MASK, !partial) && (x0 & 1) == 0 && (pitch & 1) == 0;
    }
    auto store_row_pairs = [&](int j, const C (&res)[V]) {
        if constexpr (PAIRABLE) {
            float *out = dst + (j * pitch + col0);
#pragma unroll
            for (int h = 0; h < V / 2; ++h) st_pair_pred(out + 2 * h, res[2 * h], res[2 * h + 1], pair_bits, h);
        }
    };
    // Level-0 row i (ring slot sb+k) -> registers, as pairs (paired rows only).
    auto load_row_pairs = [&](int i, int k, C (&row)[V]) -> bool {
        if constexpr (PAIRABLE) {
            if (!mbar_wait_warp(&bars[sb + k], par, status)) return false;
            const float2 *src = reinterpret_cast<const float2 *>(row_in_slot(i, sb + k));
#pragma unroll
            for (int h = 0; h < V / 2; ++h) {
                const float2 q = src[h];
                row[2 * h] = q.x, row[2 * h + 1] = q.y;
            }
        }
        return true;
    };
    // Level-0 row i (ring slot sb+k) -> registers.  Returns false on a timeout.
    auto load_row = [&](int i, int k, bool have, C (&row)[V]) -> bool {
        if (have) {
            if (!mbar_wait_warp(&bars[sb + k], par, status)) return false;
            const S *src = row_in_slot(i, sb + k);
#pragma unroll
            for (int v = 0; v < V; ++v) row[v] = load_c<S>(src[v]);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) row[v] = C(0);
        }
        return true;
    };
    // Request the P rows of the group PF rows ahead, one lane per row.
    auto prefetch_group = [&](int ib) {
        __syncwarp();
        if (lane < P) {
            const int r = ib + PF + lane;
            int s = sb + PF + lane;
            if (s >= D) s -= D;
            if (r < rend) issue(r, s);
        }
    };
    auto advance = [&]() {
        sb += P;
        if (sb == D) {
            sb = 0;
            par ^= 1u;
        }
    };
    // After a timeout: wait (bounded) for every copy this warp still has in
    // flight, so none lands in shared memory after the warp exits.
    auto drain = [&](int ib) {
        int s = sb;
        uint32_t ph = par;
        for (int r = ib; r < ib + PF + P && r < rend; ++r) {
            mbar_wait_warp(&bars[s], ph, status);
            if (++s == D) {
                s = 0;
                ph ^= 1u;
            }
        }
    };

    // FP32 plain chains run on packed pairs of cells (f32x2) wherever both
    // operands are already paired: the centre, every y-shifted row and the
    // even x-shifts.  An odd x-shift would pair cells of two different
    // pairs, so those terms run as scalar fmas on the two halves of the
    // packed accumulator.  Each half still sees exactly the canonical chain.
    constexpr bool PACKED = PACK && std::is_same<S, float>::value && MODE == MODE_PLAIN;
    constexpr int H = V / 2;

    if constexpr (SHAPE == SH_STAR && PACKED) {
        // rr[t][r % P][h] = cells 2h, 2h+1 of level-t row r, t = 0..bT-1
        f2_t rr[BT][P][H];
#pragma unroll
        for (int t = 0; t < BT; ++t)
#pragma unroll
            for (int s2 = 0; s2 < P; ++s2)
#pragma unroll
                for (int h = 0; h < H; ++h) rr[t][s2][h] = 0ull;

        auto group = [&](auto check_tag, auto edge_tag, auto pair_tag, int ib) -> bool {
            constexpr bool CHECK = decltype(check_tag)::value;
            constexpr bool EDGE = decltype(edge_tag)::value;
            constexpr bool PAIR = decltype(pair_tag)::value;
            prefetch_group(ib);
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int i = ib + k;
                if (CHECK && i >= iend) return true;
                {
                    float row[V];
                    if (PAIR ? !load_row_pairs(i, k, row) : !load_row(i, k, !CHECK || i < nrows, row))
                        return false;
#pragma unroll
                    for (int h = 0; h < H; ++h) rr[0][k][h] = f2_pack(row[2 * h], row[2 * h + 1]);
                }
#pragma unroll
                for (int t = 1; t <= BT; ++t) {
                    const int j = i - t * R;
                    const int sj = ((k - t * R) % P + P) % P;
                    if (CHECK && (j < R || j >= ny + R)) {
                        if (t < BT) {
#pragma unroll
                            for (int h = 0; h < H; ++h) rr[t][sj][h] = rr[t - 1][sj][h];
                        }
                        continue;
                    }
                    if (CHECK && t == BT && (j < y0 || j >= y1)) continue;
                    float x[V];
#pragma unroll
                    for (int h = 0; h < H; ++h) f2_unpack(rr[t - 1][sj][h], x[2 * h], x[2 * h + 1]);
                    float L[R], Rt[R];
#pragma unroll
                    for (int d = 1; d <= R; ++d) {
                        L[d - 1] = __shfl_up_sync(FULL_MASK, x[V - d], 1);
                        Rt[d - 1] = __shfl_down_sync(FULL_MASK, x[d - 1], 1);
                    }
                    f2_t acc[H];
#pragma unroll
                    for (int h = 0; h < H; ++h) acc[h] = f2_mul(cp[0], rr[t - 1][sj][h]);
                    int kk = 1;
#pragma unroll
                    for (int ii = -R; ii <= R; ++ii) {
                        if (ii == 0) continue;
                        // x-shift ii: even and inside the lane -> packed; else scalar halves
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            const int m = 2 * h + ii;
                            if (ii % 2 == 0 && m >= 0 && m + 1 < V) {
                                acc[h] = f2_fma(cp[kk], rr[t - 1][sj][m / 2], acc[h]);
                            } else {
                                float lo, hi;
                                f2_unpack(acc[h], lo, hi);
                                const float x0 = m < 0 ? L[-m - 1] : (m >= V ? Rt[m - V] : x[m]);
                                const float x1 =
                                    m + 1 < 0 ? L[-m - 2] : (m + 1 >= V ? Rt[m + 1 - V] : x[m + 1]);
                                lo = op_fma(cf[kk], x0, lo);
                                hi = op_fma(cf[kk], x1, hi);
                                acc[h] = f2_pack(lo, hi);
                            }
                        }
                        const int sy = ((k - t * R + ii) % P + P) % P;
#pragma unroll
                        for (int h = 0; h < H; ++h) acc[h] = f2_fma(cp[kk + 1], rr[t - 1][sy][h], acc[h]);
                        kk += 2;
                    }
                    if constexpr (POST != POST_NONE) {
#pragma unroll
                        for (int h = 0; h < H; ++h) acc[h] = f2_post<POST>(acc[h], post_p, post_c);
                    }
                    if (t < BT) {
                        if (EDGE) {
#pragma unroll
                            for (int h = 0; h < H; ++h) {
                                float r0, r1;
                                f2_unpack(acc[h], r0, r1);
                                if (halo_bits & (1u << (2 * h))) r0 = x[2 * h];
                                if (halo_bits & (1u << (2 * h + 1))) r1 = x[2 * h + 1];
                                acc[h] = f2_pack(r0, r1);
                            }
                        }
#pragma unroll
                        for (int h = 0; h < H; ++h) rr[t][sj][h] = acc[h];
                    } else {
                        float res[V];
#pragma unroll
                        for (int h = 0; h < H; ++h) f2_unpack(acc[h], res[2 * h], res[2 * h + 1]);
                        if (PAIR)
                            store_row_pairs(j, res);
                        else
                            store_row(j, res);
                    }
                }
            }
            return true;
        };

        for (int ib = ib0; ib < iend; ib += P) {
            const bool fast = (ib - BT * R >= y0) && (ib + P - 1 - BT * R < y1) &&
                              (ib - BT * R >= R) && (ib + P - 1 - R < ny + R);
            bool ok;
            if (fast && edge)
                ok = group(std::false_type{}, std::true_type{}, std::false_type{}, ib);
            else if (fast && paired)
                ok = group(std::false_type{}, std::false_type{}, std::true_type{}, ib);
            else if (fast)
                ok = group(std::false_type{}, std::false_type{}, std::false_type{}, ib);
            else
                ok = group(std::true_type{}, std::true_type{}, std::false_type{}, ib);
            if (!ok) {
                drain(ib);
                return false;
            }
            advance();
        }
    } else if constexpr (SHAPE == SH_BOX && PACKED) {
        // pa[t-1][r % P][h] = pending partial sums of cells 2h, 2h+1 of level-t row r
        f2_t pa[BT][P][H];
#pragma unroll
        for (int t = 0; t < BT; ++t)
#pragma unroll
            for (int s2 = 0; s2 < P; ++s2)
#pragma unroll
                for (int h = 0; h < H; ++h) pa[t][s2][h] = 0ull;

        auto group = [&](auto check_tag, auto edge_tag, auto pair_tag, int ib) -> bool {
            constexpr bool CHECK = decltype(check_tag)::value;
            constexpr bool EDGE = decltype(edge_tag)::value;
            constexpr bool PAIR = decltype(pair_tag)::value;
            prefetch_group(ib);
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int i = ib + k;
                if (CHECK && i >= iend) return true;
                float in_row[V];
                if (PAIR ? !load_row_pairs(i, k, in_row) : !load_row(i, k, !CHECK || i < nrows, in_row))
                    return false;
#pragma unroll
                for (int t = 1; t <= BT; ++t) {
                    const int ar = i - (t - 1) * R;
                    // even x-shifts as pairs: XE[q + R/2] = cells 2q, 2q+1 (q may reach into
                    // the neighbouring lanes); odd shifts use the scalar extended row e
                    float e[V + 2 * R];
#pragma unroll
                    for (int v = 0; v < V; ++v) e[R + v] = in_row[v];
#pragma unroll
                    for (int d = 1; d <= R; ++d) {
                        e[R - d] = __shfl_up_sync(FULL_MASK, in_row[V - d], 1);
                        e[R + V - 1 + d] = __shfl_down_sync(FULL_MASK, in_row[d - 1], 1);
                    }
                    constexpr int QL = R / 2;  // pairs needed beyond each side for even shifts
                    f2_t XE[H + 2 * QL];
#pragma unroll
                    for (int q = -QL; q < H + QL; ++q)
                        XE[q + QL] = f2_pack(e[R + 2 * q], e[R + 2 * q + 1]);
#pragma unroll
                    for (int dy = -R; dy <= R; ++dy) {
                        const int b = ar - dy;
                        const int sp = ((k - (t - 1) * R - dy) % P + P) % P;
                        if (CHECK && (b < R || b >= ny + R)) {
                            if (dy == 0 && t < BT) {
#pragma unroll
                                for (int h = 0; h < H; ++h) pa[t - 1][sp][h] = XE[h + QL];
                            }
                            continue;
                        }
#pragma unroll
                        for (int dx = -R; dx <= R; ++dx) {
                            const int kk = (dy + R) * P + (dx + R);
                            const bool first = (dy == -R && dx == -R);
#pragma unroll
                            for (int h = 0; h < H; ++h) {
                                if (dx % 2 == 0) {
                                    const f2_t xv = XE[h + dx / 2 + QL];
                                    pa[t - 1][sp][h] = first ? f2_mul(cp[kk], xv)
                                                             : f2_fma(cp[kk], xv, pa[t - 1][sp][h]);
                                } else {
                                    const float x0 = e[R + 2 * h + dx], x1 = e[R + 2 * h + dx + 1];
                                    float lo, hi;
                                    if (first) {
                                        lo = op_mul(cf[kk], x0);
                                        hi = op_mul(cf[kk], x1);
                                    } else {
                                        f2_unpack(pa[t - 1][sp][h], lo, hi);
                                        lo = op_fma(cf[kk], x0, lo);
                                        hi = op_fma(cf[kk], x1, hi);
                                    }
                                    pa[t - 1][sp][h] = f2_pack(lo, hi);
                                }
                            }
                        }
                    }
                    const int e_row = i - t * R;
                    const int se = ((k - t * R) % P + P) % P;
                    // a halo row's pending value is its fixed copy: no per-step division
                    const bool inner = !CHECK || (e_row >= R && e_row < ny + R);
                    float out_row[V];
#pragma unroll
                    for (int h = 0; h < H; ++h)
                        f2_unpack(inner ? f2_post<POST>(pa[t - 1][se][h], post_p, post_c) : pa[t - 1][se][h],
                                  out_row[2 * h], out_row[2 * h + 1]);
                    if (t < BT) {
                        if (EDGE) {
                            int s2 = sb + (k - t * R);
                            if (s2 < 0) s2 += D;
                            const float *orig = row_in_slot(e_row, s2);
#pragma unroll
                            for (int v = 0; v < V; ++v)
                                if (halo_bits & (1u << v)) out_row[v] = orig[v];
                        }
#pragma unroll
                        for (int v = 0; v < V; ++v) in_row[v] = out_row[v];
                    } else if (!CHECK || (e_row >= y0 && e_row < y1)) {
                        if (PAIR)
                            store_row_pairs(e_row, out_row);
                        else
                            store_row(e_row, out_row);
                    }
                }
            }
            return true;
        };

        for (int ib = ib0; ib < iend; ib += P) {
            const bool fast = (ib - BT * R >= y0) && (ib + P - 1 - BT * R < y1) &&
                              (ib - BT * R >= R) && (ib + P - 1 + R < ny + R);
            bool ok;
            if (fast && edge)
                ok = group(std::false_type{}, std::true_type{}, std::false_type{}, ib);
            else if (fast && paired)
                ok = group(std::false_type{}, std::false_type{}, std::true_type{}, ib);
            else if (fast)
                ok = group(std::false_type{}, std::false_type{}, std::false_type{}, ib);
            else
                ok = group(std::true_type{}, std::true_type{}, std::false_type{}, ib);
            if (!ok) {
                drain(ib);
                return false;
            }
            advance();
        }
    } else if constexpr (SHAPE == SH_STAR) {
        // rr[t][r % P] = level-t row r, t = 0..bT-1
        C rr[BT][P][V];
#pragma unroll
        for (int t = 0; t < BT; ++t)
#pragma unroll
            for (int s = 0; s < P; ++s)
#pragma unroll
                for (int v = 0; v < V; ++v) rr[t][s][v] = C(0);

        auto group = [&](auto check_tag, auto edge_tag, int ib) -> bool {
            constexpr bool CHECK = decltype(check_tag)::value;
            constexpr bool EDGE = decltype(edge_tag)::value;
            prefetch_group(ib);
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int i = ib + k;
                if (CHECK && i >= iend) return true;
                if (!load_row(i, k, !CHECK || i < nrows, rr[0][k])) return false;
                if constexpr (HOOK::active)
                    if (!CHECK || (i >= R && i < ny + R)) hook->row(0, i, rr[0][k]);
#pragma unroll
                for (int t = 1; t <= BT; ++t) {
                    const int j = i - t * R;  // level-t row completed now
                    const int sj = ((k - t * R) % P + P) % P;
                    if (CHECK && (j < R || j >= ny + R)) {  // halo row: fixed value
                        if (t < BT) {
#pragma unroll
                            for (int v = 0; v < V; ++v) rr[t][sj][v] = rr[t - 1][sj][v];
                        }
                        continue;
                    }
                    if (CHECK && t == BT && (j < y0 || j >= y1)) continue;
                    C L[R], Rt[R];
                    exchange(rr[t - 1][sj], L, Rt);
                    Acc<MODE, C> acc[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[v].first(cf[0], rr[t - 1][sj][v]);
                    int kk = 1;
#pragma unroll
                    for (int ii = -R; ii <= R; ++ii) {
                        if (ii == 0) continue;
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const int s = v + ii;
                            const C xv = s < 0 ? L[-s - 1] : (s >= V ? Rt[s - V] : rr[t - 1][sj][s]);
                            acc[v].add(cf[kk], xv);
                        }
                        const int sy = ((k - t * R + ii) % P + P) % P;
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v].add(cf[kk + 1], rr[t - 1][sy][v]);
                        kk += 2;
                    }
                    C res[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) res[v] = level_round<S>(post_op<POST>(acc[v].result(), post_c));
                    if (t < BT) {
                        if (EDGE) {
#pragma unroll
                            for (int v = 0; v < V; ++v)
                                if (halo_bits & (1u << v)) res[v] = rr[t - 1][sj][v];
                        }
#pragma unroll
                        for (int v = 0; v < V; ++v) rr[t][sj][v] = res[v];
                        if (LEVELS && j >= y0 && j < y1) store_row_to(lvl[t], j, res);
                        if constexpr (HOOK::active) hook->row(t, j, res);
                    } else {
                        store_row(j, res);
                    }
                }
            }
            return true;
        };

        for (int ib = ib0; ib < iend; ib += P) {
            // fast: every row of the group is interior at every level and
            // every level-bT row it completes is stored by this warp
            const bool fast = (ib - BT * R >= y0) && (ib + P - 1 - BT * R < y1) &&
                              (ib - BT * R >= R) && (ib + P - 1 - R < ny + R);
            bool ok;
            if (fast)
                ok = edge ? group(std::false_type{}, std::true_type{}, ib)
                          : group(std::false_type{}, std::false_type{}, ib);
            else
                ok = group(std::true_type{}, std::true_type{}, ib);
            if (!ok) {
                drain(ib);
                return false;
            }
            advance();
        }
    } else {
        // pa[t-1][r % P] = pending partial sum of level-t row r, t = 1..bT
        Acc<MODE, C> pa[BT][P][V];
#pragma unroll
        for (int t = 0; t < BT; ++t)
#pragma unroll
            for (int s = 0; s < P; ++s)
#pragma unroll
                for (int v = 0; v < V; ++v) pa[t][s][v].set(C(0));

        auto group = [&](auto check_tag, auto edge_tag, int ib) -> bool {
            constexpr bool CHECK = decltype(check_tag)::value;
            constexpr bool EDGE = decltype(edge_tag)::value;
            prefetch_group(ib);
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int i = ib + k;
                if (CHECK && i >= iend) return true;
                C in_row[V];
                if (!load_row(i, k, !CHECK || i < nrows, in_row)) return false;
                if constexpr (HOOK::active)
                    if (!CHECK || (i >= R && i < ny + R)) hook->row(0, i, in_row);
#pragma unroll
                for (int t = 1; t <= BT; ++t) {
                    const int ar = i - (t - 1) * R;  // arriving level-(t-1) row
                    C L[R], Rt[R];
                    exchange(in_row, L, Rt);
#pragma unroll
                    for (int dy = -R; dy <= R; ++dy) {
                        const int b = ar - dy;  // pending level-t row receiving its dy term
                        const int sp = ((k - (t - 1) * R - dy) % P + P) % P;
                        if (CHECK && (b < R || b >= ny + R)) {
                            if (dy == 0 && t < BT) {
#pragma unroll
                                for (int v = 0; v < V; ++v) pa[t - 1][sp][v].set(in_row[v]);
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
                                    pa[t - 1][sp][v].first(cf[kk], xv);
                                else
                                    pa[t - 1][sp][v].add(cf[kk], xv);
                            }
                        }
                    }
                    const int e = i - t * R;  // level-t row completed now
                    const int se = ((k - t * R) % P + P) % P;
                    C out_row[V];
                    // a halo row's pending value is its fixed copy: no per-step division
                    const bool inner = !CHECK || (e >= R && e < ny + R);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const C x = pa[t - 1][se][v].result();
                        out_row[v] = level_round<S>(inner ? post_op<POST>(x, post_c) : x);
                    }
                    if (t < BT) {
                        if (EDGE) {
                            // input value of row e, still in its ring slot k - t*R slots back
                            int s = sb + (k - t * R);
                            if (s < 0) s += D;
                            const S *orig = row_in_slot(e, s);
#pragma unroll
                            for (int v = 0; v < V; ++v)
                                if (halo_bits & (1u << v)) out_row[v] = load_c<S>(orig[v]);
                        }
#pragma unroll
                        for (int v = 0; v < V; ++v) in_row[v] = out_row[v];
                        if (LEVELS && e >= y0 && e < y1) store_row_to(lvl[t], e, out_row);
                        if constexpr (HOOK::active)
                            if (inner) hook->row(t, e, out_row);
                    } else if (!CHECK || (e >= y0 && e < y1)) {
                        store_row(e, out_row);
                    }
                }
            }
            return true;
        };

        for (int ib = ib0; ib < iend; ib += P) {
            const bool fast = (ib - BT * R >= y0) && (ib + P - 1 - BT * R < y1) &&
                              (ib - BT * R >= R) && (ib + P - 1 + R < ny + R);
            bool ok;
            if (fast)
                ok = edge ? group(std::false_type{}, std::true_type{}, ib)
                          : group(std::false_type{}, std::false_type{}, ib);
            else
                ok = group(std::true_type{}, std::true_type{}, ib);
            if (!ok) {
                drain(ib);
                return false;
            }
            advance();
        }
    }
    return true;
}

// OCC_ > 0 fixes the CTAs per SM the registers are sized for (else the
// Sweep2DOccupancy estimate).
template <int SHAPE, int R, int BT, typename S, int MODE, int POST, int V_, int OCC_>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32,
                                  (OCC_ > 0 ? OCC_ : Sweep2DOccupancy<S, SHAPE, BT, R, MODE, V_>::value))
    sweep2d_kernel(const __grid_constant__ CUtensorMap tmap,
                   const Sweep2DArgs<S, NCoeff2<SHAPE, R>::value> a)
{
    using G = Sweep2DGeom<S, BT, R, V_>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * WARPS_PER_CTA + warp;
    if (gw >= a.total_warps) return;
    // tile geometry (Section 3.1): tiles advance by the compute-region width,
    // each starting bT*R cells left of its compute region
    const int xt = gw % a.tiles_x;
    const int sbk = gw / a.tiles_x;
    Tile2D tg;
    tg.src = nullptr;
    tg.total = 0;
    tg.pitch = a.pitch;
    tg.ny = a.ny;
    tg.nx = a.nx;
    tg.x0 = a.xb0 - BT * R + xt * a.tile_stride;
    tg.sc0 = max(R, tg.x0 + BT * R);
    tg.sc1 = min(a.nx + R, tg.x0 + BT * R + a.tile_stride);
    tg.y0 = R + sbk * a.hsn;
    tg.y1 = min(tg.y0 + a.hsn, a.ny + R);
    tg.stall = a.stall_test && gw == 0;
    // Box chains address the rings through a pointer derived from the shared
    // array by arithmetic (the compiler then keeps their accesses in the
    // shared address space); star chains through the generic round trip,
    // which measured faster for them.
    unsigned char *const smem_al =
        SHAPE == SH_BOX ? smem + ((128u - (smem_u32(smem) & 127u)) & 127u)
                        : reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem) + 127) & ~uintptr_t(127));
    // Boxes of radius 2 and more run the scalar chain: with (2R+1)^2 terms the
    // odd x shifts (scalar fmas on repacked halves) outnumber the paired
    // terms, and the plain chain with constant-bank coefficients measured
    // 1-3% faster (box2d2r-box2d4r).
    constexpr bool PACK_CHAIN = !(SHAPE == SH_BOX && R >= 2);
    sweep2d_tile<SHAPE, R, BT, S, MODE, PACK_CHAIN, decltype(a.k.c), decltype(a.kp.c), false, false, POST, V_>(
        tg, &tmap, a.dst, a.status, smem_al + warp * G::WARP_BYTES, a.k.c, a.kp.c, nullptr, a.post_c,
        a.post_p);
}

// Host-side launcher of one instantiation.
template <int SHAPE, int R, int BT, typename S, int MODE, int POST, int V_, int OCC_>
cudaError_t launch_sweep2d(const PassDesc &d, cudaStream_t st)
{
    constexpr int N = NCoeff2<SHAPE, R>::value;
    using C = typename StorageTraits<S>::C;
    using G = Sweep2DGeom<S, BT, R, V_>;
    // the descriptor must describe this kernel's tile width (its TMA box too)
    if (d.tile_stride_x != G::TILE - 2 * BT * R) return cudaErrorInvalidValue;
    Sweep2DArgs<S, N> a;
    a.dst = static_cast<S *>(d.dst);
    a.status = d.status;
    a.pitch = static_cast<int>(d.pitch);
    a.ny = d.ny;
    a.nx = d.nx;
    a.tile_stride = d.tile_stride_x;
    a.xb0 = d.x_base;
    a.tiles_x = d.tiles_x;
    a.hsn = d.hsn;
    a.total_warps = d.total_units;
    a.stall_test = d.stall_test;
    for (int k = 0; k < N; ++k) {
        a.k.c[k] = static_cast<C>(d.coeffs[k]);
        const float f = static_cast<float>(d.coeffs[k]);
        unsigned u;
        memcpy(&u, &f, 4);
        a.kp.c[k] = ((unsigned long long)u << 32) | u;
    }
    a.post_c = static_cast<C>(d.post_c);
    {
        const float f = static_cast<float>(d.post_c);
        unsigned u;
        memcpy(&u, &f, 4);
        a.post_p = ((unsigned long long)u << 32) | u;
    }
    auto fn = sweep2d_kernel<SHAPE, R, BT, S, MODE, POST, V_, OCC_>;
    if (G::CTA_BYTES > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             G::CTA_BYTES);
        if (e != cudaSuccess) return e;
    }
    fn<<<d.ctas, WARPS_PER_CTA * 32, G::CTA_BYTES, st>>>(d.tmap, a);
    return cudaGetLastError();
}

// V_ = cells per lane: the default width registers as tile variant 0, a
// wider one under its tile width (32 * V_ cells).
template <int SHAPE, int R, int BT, typename S, int MODE, int POST = POST_NONE, int V_ = CELLS_PER_LANE,
          int OCC_ = 0>
KernelEntry entry2d(int dtype)
{
    using G = Sweep2DGeom<S, BT, R, V_>;
    KernelEntry e;
    e.key = KernelKey{2, SHAPE, R, dtype, BT, POST, V_ == CELLS_PER_LANE ? 0 : G::TILE};
    e.launch = &launch_sweep2d<SHAPE, R, BT, S, MODE, POST, V_, OCC_>;
    e.func = reinterpret_cast<const void *>(&sweep2d_kernel<SHAPE, R, BT, S, MODE, POST, V_, OCC_>);
    e.threads = WARPS_PER_CTA * 32;
    e.smem_bytes = G::CTA_BYTES;
    e.tile_x = G::TILE;
    e.tile_y = 1;
    e.units_per_cta = WARPS_PER_CTA;
    return e;
}

}  // namespace an5d
