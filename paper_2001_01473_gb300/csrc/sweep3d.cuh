// sweep3d.cuh -- 2.5D-blocked, temporally blocked 3D stencil sweep (sm_103a).
//
// Method (AN5D, Section 3.1, Fig. 1; Section 3.2): tile the y and x axes,
// stream along z, fuse bT time levels per pass; level t lags level t-1 by R
// planes and its valid region shrinks by R cells per side in y and x; only
// level bT's compute region is stored.  The z axis is cut into stream blocks
// of hsn planes (Section 3.2, division of the streaming dimension).
//
// GB300 mapping (this library's design):
//  * a CTA of NW warps owns a tile of TY = RW*NW rows (y) by TX = 32*V cells
//    (x); each warp owns RW rows, each lane V consecutive x cells of them
//    (V = 4, RW = 2 by default; V = 2, RW = 4 gives 64-cell-wide tiles);
//  * input planes are staged by TMA into a shared-memory ring of planes:
//    each warp copies its own rows (one 1D row copy per lane) and waits on
//    its own mbarrier per ring slot, so no warp serialises a whole plane's
//    copies and the ring needs no CTA-wide synchronisation;
//  * each level keeps the 2R+1 most recent planes of the thread's 8 cells
//    (star) or 2R+1 pending per-plane partial sums (box) in registers, in a
//    fixed ring indexed by plane mod (2R+1) (Section 3.2 register allocation);
//  * x neighbours travel by warp shuffles; y neighbours owned by other warps
//    go through a double-buffered shared-memory exchange of the level's
//    plane rows with one CTA barrier per level and plane (Section 3.2,
//    shared-memory double buffering);
//  * Dirichlet halo: halo planes are copied level to level; in tiles that
//    touch the domain boundary, halo cells are reset to their input values
//    after every level (Section 3.1).
#pragma once

#include <cstring>
#include <type_traits>

#include "an5d_internal.h"
#include "device_common.cuh"

namespace an5d {

// V cells of a lane to or from the y-exchange buffer.  Each lane's cells
// start on a 16-byte boundary there (128-byte aligned buffer, rows of
// 32 * V cells), so whole 16-byte vectors move where V cells fill them.
template <typename C, int V> __device__ __forceinline__ void xb_store(C *p, const C (&v)[V])
{
    if constexpr (std::is_same<C, float>::value && V % 4 == 0) {
#pragma unroll
        for (int i = 0; i < V / 4; ++i)
            reinterpret_cast<float4 *>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (std::is_same<C, double>::value && V % 2 == 0) {
#pragma unroll
        for (int i = 0; i < V / 2; ++i) reinterpret_cast<double2 *>(p)[i] = make_double2(v[2 * i], v[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) p[i] = v[i];
    }
}
template <typename C, int V> __device__ __forceinline__ void xb_load(const C *p, C (&v)[V])
{
    if constexpr (std::is_same<C, float>::value && V % 4 == 0) {
#pragma unroll
        for (int i = 0; i < V / 4; ++i) {
            const float4 q = reinterpret_cast<const float4 *>(p)[i];
            v[4 * i] = q.x, v[4 * i + 1] = q.y, v[4 * i + 2] = q.z, v[4 * i + 3] = q.w;
        }
    } else if constexpr (std::is_same<C, double>::value && V % 2 == 0) {
#pragma unroll
        for (int i = 0; i < V / 2; ++i) {
            const double2 q = reinterpret_cast<const double2 *>(p)[i];
            v[2 * i] = q.x, v[2 * i + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) v[i] = p[i];
    }
}

template <int SHAPE, int R> struct NCoeff3 {
    static constexpr int value = SHAPE == SH_STAR ? 6 * R + 1 : (2 * R + 1) * (2 * R + 1) * (2 * R + 1);
};

template <typename S, int N> struct Sweep3DArgs {
    S *dst;
    int *status;
    int px;           // padded row length nx + 2R
    int py;           // padded rows per plane ny + 2R
    int nz, ny, nx;   // interior extents
    int tsx, tsy;     // output columns / rows per tile
    int xb0;          // padded column where tile column 0's compute region starts
    int tiles_x, tiles_y;
    int hsn;          // output planes per stream block
    int total_ctas;   // tiles_x * tiles_y * stream blocks
    CoeffBlock<typename StorageTraits<S>::C, N> k;
    typename StorageTraits<S>::C post_c;  // divisor or reciprocal (division-type stencils)
};

template <typename S, int SHAPE, int BT, int R, int NW, int V_ = CELLS_PER_LANE, int RW_ = 2>
struct Sweep3DGeom {
    static constexpr int V = V_;                 // consecutive x cells per lane
    static constexpr int RW = RW_;               // rows per warp
    static constexpr int TY = NW * RW;           // tile rows
    static constexpr int TX = 32 * V;            // tile columns
    static constexpr int P = 2 * R + 1;
    static constexpr int A = StorageTraits<S>::ALIGN_ELEMS;
    static constexpr int ROWBUF = TX + A;        // TMA box per row
    static constexpr int ROW_BYTES = ((ROWBUF * (int)sizeof(S) + 127) / 128) * 128;
    static constexpr int SLOT_BYTES = TY * ROW_BYTES;
    // box edge tiles re-read halo cells of planes up to bT*R behind
    static constexpr int KEEP = SHAPE == SH_BOX ? BT * R : 0;
    using C = typename StorageTraits<S>::C;
    static constexpr int XB_BYTES = 2 * TY * TX * (int)sizeof(C);  // y-exchange, double buffered
    // Planes in flight ahead of the consumer: as many as shared memory holds,
    // between PREFETCH_ROWS and 6 (one CTA per SM keeps only this CTA's
    // copies in flight, so a deeper ring hides more of the DRAM latency).
    static constexpr int PF_FIT = (232448 - 128 - XB_BYTES) / (SLOT_BYTES + NW * 8) - KEEP - 1;
    static constexpr int PF = PF_FIT > 6 ? 6 : (PF_FIT < PREFETCH_ROWS ? PREFETCH_ROWS : PF_FIT);
    static constexpr int D = PF + KEEP + 1;                        // ring depth (planes)
    static constexpr int SMEM_BYTES = D * SLOT_BYTES + XB_BYTES + D * NW * 8 + 128;
    static_assert(SMEM_BYTES <= 232448, "shared memory per CTA exceeds 227 KB");
    static_assert(TX - 2 * BT * R >= 8 && TY - 2 * BT * R >= 2, "tile too small for bT*R");
    static_assert(R <= V, "radius must not exceed cells per lane");
    static_assert(RW * V <= 32, "cell bit masks");
};

template <int SHAPE, int R, int BT, typename S, int MODE, int NW, int POST, int V_, int RW_>
__global__ void __launch_bounds__(NW * 32, 1)
    sweep3d_kernel(const __grid_constant__ CUtensorMap tmap,
                   const Sweep3DArgs<S, NCoeff3<SHAPE, R>::value> a)
{
    using C = typename StorageTraits<S>::C;
    using G = Sweep3DGeom<S, SHAPE, BT, R, NW, V_, RW_>;
    constexpr int V = G::V, RW = G::RW, TY = G::TY, TX = G::TX, P = G::P, D = G::D, A = G::A,
                  PF = G::PF;
    extern __shared__ __align__(128) unsigned char smem[];

    const int cta = blockIdx.x;
    if (cta >= a.total_ctas) return;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    // ---- tile geometry ----
    const int xt = cta % a.tiles_x;
    const int yt = (cta / a.tiles_x) % a.tiles_y;
    const int zb = cta / (a.tiles_x * a.tiles_y);
    const int x0 = a.xb0 - BT * R + xt * a.tsx;   // padded column of the tile's first cell
    const int yb = R - BT * R + yt * a.tsy;   // padded row of the tile's first row
    const int px = a.px, py = a.py, nz = a.nz, ny = a.ny, nx = a.nx;
    const int nplanes = nz + 2 * R;
    const int z0 = R + zb * a.hsn;
    const int z1 = min(z0 + a.hsn, nz + R);
    const int zs = max(0, z0 - BT * R);
    const int ib0 = zs - zs % P;
    const int iend = z1 + BT * R;
    const int pend = min(nplanes, iend);       // planes requested: exactly the planes consumed

    const int col0 = x0 + lane * V;
    const int row0 = yb + warp * RW;          // padded row of this warp's first row
    const int sc0 = max(R, x0 + BT * R), sc1 = min(nx + R, x0 + BT * R + a.tsx);
    const int sr0 = max(R, yb + BT * R), sr1 = min(ny + R, yb + BT * R + a.tsy);
    unsigned halo_bits = 0, store_bits = 0;   // bit r*V+v
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int y = row0 + r, x = col0 + v;
            if (y < R || y >= ny + R || x < R || x >= nx + R) halo_bits |= 1u << (r * V + v);
            if (y >= sr0 && y < sr1 && x >= sc0 && x < sc1) store_bits |= 1u << (r * V + v);
        }
    const bool edge = __syncthreads_or(halo_bits != 0) != 0;

    // aligned by pointer arithmetic on the shared array, so that the compiler
    // keeps the staged-row and exchange accesses in the shared address space
    unsigned char *const base = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    unsigned char *const ring = base;
    C *const xb = reinterpret_cast<C *>(base + D * G::SLOT_BYTES);
    uint64_t *const bars = reinterpret_cast<uint64_t *>(base + D * G::SLOT_BYTES + G::XB_BYTES);
    int *const status = a.status;

    // Every warp stages its own RW rows of each plane (lane r copies row
    // warp*RW + r) and waits on its own mbarrier per slot: a warp reads only
    // its own staged rows, so the ring needs no CTA-wide synchronisation, and
    // no single warp serialises the plane's row copies.
    int nissue = ib0;  // next plane this warp requests
    auto issue_plane = [&](int p, int s) {
        if (lane == 0) mbar_expect_tx(&bars[s * NW + warp], RW * G::ROWBUF * (int)sizeof(S));
        __syncwarp();
        // No proxy fence before the copy: the slot's previous rows were read
        // by this warp only, and those reads completed (their values were
        // used) iterations before the slot is refilled.
        if (lane < RW) {
            const int row = warp * RW + lane;
            const int lin = (p * py + yb + row) * px + x0;
            tma_load_1d(ring + s * G::SLOT_BYTES + row * G::ROW_BYTES, &tmap, lin & ~(A - 1),
                        &bars[s * NW + warp]);
        }
        nissue = p + 1;
    };
    // This thread's cells of tile row (warp*RW + r) of plane p in slot s.
    auto cells_in_slot = [&](int p, int s, int r) -> const S * {
        const int lin = (p * py + row0 + r) * px + x0;
        return reinterpret_cast<const S *>(ring + s * G::SLOT_BYTES + (warp * RW + r) * G::ROW_BYTES) +
               (lin & (A - 1)) + lane * V;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < D * NW; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    for (int q = 0; q < PF; ++q)
        if (ib0 + q < pend) issue_plane(ib0 + q, q);

    // Ring position of plane cur_p: slot cs, mbarrier phase cpar.
    int cs = 0, cur_p = ib0;
    uint32_t cpar = 0;
    int xsel = 0;        // exchange buffer in use
    // First plane whose wait gave up, with its slot and phase (-1: none).
    int fpl = -1, fcs = 0;
    uint32_t fpar = 0;

    const auto &cf = a.k.c;
    S *const dst = a.dst;

    // Start of iteration i: request plane i+PF (its slot last held plane
    // i+PF-D, whose rows of this warp it has read already), then wait for
    // plane i and copy this thread's cells to registers.  After a wait gives
    // up the warp stops requesting planes and keeps computing on zeros, so
    // that every CTA barrier of the group is still reached; the pass's
    // result is then discarded (the plan's status reports the timeout).
    auto load_plane = [&](int i, bool have, C (&cell)[RW][V], bool &ok) {
        if (ok && i + PF < pend) {
            int s = cs + PF;
            if (s >= D) s -= D;
            issue_plane(i + PF, s);
        }
        if (have && ok) {
            ok = mbar_wait_warp(&bars[cs * NW + warp], cpar, status);
            if (!ok) {
                fpl = i;
                fcs = cs;
                fpar = cpar;
            }
        }
        if (have && ok) {
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                load_cells<S, V>(cells_in_slot(i, cs, r), cell[r]);
            }
        } else {
#pragma unroll
            for (int r = 0; r < RW; ++r)
#pragma unroll
                for (int v = 0; v < V; ++v) cell[r][v] = C(0);
        }
    };
    auto advance = [&]() {
        ++cur_p;
        if (++cs == D) {
            cs = 0;
            cpar ^= 1u;
        }
    };
    // After a timeout anywhere in the CTA every warp leaves; first it waits
    // (bounded) for its own copies still in flight, from the first plane it
    // has not consumed (or the one whose wait gave up) to the last it
    // requested, so that none lands after the CTA exits.
    auto drain = [&](int) {
        int p0 = cur_p, s = cs;
        uint32_t ph = cpar;
        if (fpl >= 0) p0 = fpl, s = fcs, ph = fpar;
        for (int p = p0; p < nissue; ++p) {
            if (!mbar_wait_warp(&bars[s * NW + warp], ph, status)) break;
            if (++s == D) {
                s = 0;
                ph ^= 1u;
            }
        }
    };
    // Publish this warp's rows of a plane, then return the tile rows
    // warp*RW - R .. warp*RW + RW - 1 + R (own rows from registers).  Rows
    // outside the tile read a clamped row: they only feed cells outside the
    // valid region.
    auto exchange = [&](const C (&own)[RW][V], C (&ext)[RW + 2 * R][V]) {
        C *buf = xb + xsel * (TY * TX);
        xsel ^= 1;
#pragma unroll
        for (int r = 0; r < RW; ++r) xb_store<C, V>(buf + (warp * RW + r) * TX + lane * V, own[r]);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < RW + 2 * R; ++q) {
            const int tr = warp * RW - R + q;  // tile row
            if (q >= R && q < R + RW) {
#pragma unroll
                for (int v = 0; v < V; ++v) ext[q][v] = own[q - R][v];
            } else {
                const int cr = tr < 0 ? 0 : (tr >= TY ? TY - 1 : tr);
                xb_load<C, V>(buf + cr * TX + lane * V, ext[q]);
            }
        }
    };
    auto store_cells = [&](int p, const C (&res)[RW][V]) {
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            S *out = dst + ((p * py + row0 + r) * px + col0);
#pragma unroll
            for (int v = 0; v < V; ++v) st_pred<S>(out + v, to_storage<S>(res[r][v]), store_bits, r * V + v);
        }
    };
    // x-shifted value of tile-relative cell v+dx of a row held as V values per lane
    auto xshift = [&](const C (&row)[V], C (&L)[R], C (&Rt)[R]) {
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            L[d - 1] = __shfl_up_sync(FULL_MASK, row[V - d], 1);
            Rt[d - 1] = __shfl_down_sync(FULL_MASK, row[d - 1], 1);
        }
    };

    if constexpr (SHAPE == SH_STAR) {
        // ring[t][p % P][r][v] = level-t plane p at this thread's cells, t = 0..bT-1
        C ring[BT][P][RW][V];
#pragma unroll
        for (int t = 0; t < BT; ++t)
#pragma unroll
            for (int s = 0; s < P; ++s)
#pragma unroll
                for (int r = 0; r < RW; ++r)
#pragma unroll
                    for (int v = 0; v < V; ++v) ring[t][s][r][v] = C(0);

        auto group = [&](auto check_tag, auto edge_tag, int ib) -> bool {
            constexpr bool CHECK = decltype(check_tag)::value;
            constexpr bool EDGE = decltype(edge_tag)::value;
            bool ok = true;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int i = ib + k;
                if (CHECK && i >= iend) return ok;
                if (CHECK) __syncthreads();  // iterations of halo planes may have no exchange
                load_plane(i, !CHECK || i < nplanes, ring[0][k], ok);
#pragma unroll
                for (int t = 1; t <= BT; ++t) {
                    const int j = i - t * R;  // level-t plane completed now
                    const int sj = ((k - t * R) % P + P) % P;
                    if (CHECK && (j < R || j >= nz + R)) {  // halo plane: fixed value
                        if (t < BT) {
#pragma unroll
                            for (int r = 0; r < RW; ++r)
#pragma unroll
                                for (int v = 0; v < V; ++v) ring[t][sj][r][v] = ring[t - 1][sj][r][v];
                        }
                        continue;
                    }
                    if (CHECK && t == BT && (j < z0 || j >= z1)) continue;
                    C ext[RW + 2 * R][V];
                    exchange(ring[t - 1][sj], ext);
                    C res[RW][V];
#pragma unroll
                    for (int r = 0; r < RW; ++r) {
                        C L[R], Rt[R];
                        xshift(ring[t - 1][sj][r], L, Rt);
                        Acc<MODE, C> acc[V];
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v].first(cf[0], ring[t - 1][sj][r][v]);
                        int kk = 1;
#pragma unroll
                        for (int ii = -R; ii <= R; ++ii) {
                            if (ii == 0) continue;
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                const int s = v + ii;
                                const C xv = s < 0 ? L[-s - 1] : (s >= V ? Rt[s - V] : ring[t - 1][sj][r][s]);
                                acc[v].add(cf[kk], xv);                        // dx = ii
                            }
#pragma unroll
                            for (int v = 0; v < V; ++v) acc[v].add(cf[kk + 1], ext[R + r + ii][v]);  // dy = ii
                            const int sz = ((k - t * R + ii) % P + P) % P;
#pragma unroll
                            for (int v = 0; v < V; ++v) acc[v].add(cf[kk + 2], ring[t - 1][sz][r][v]);  // dz = ii
                            kk += 3;
                        }
#pragma unroll
                        for (int v = 0; v < V; ++v)
                            res[r][v] = level_round<S>(post_op<POST>(acc[v].result(), a.post_c));
                    }
                    if (t < BT) {
                        if (EDGE) {
#pragma unroll
                            for (int r = 0; r < RW; ++r)
#pragma unroll
                                for (int v = 0; v < V; ++v)
                                    if (halo_bits & (1u << (r * V + v))) res[r][v] = ring[t - 1][sj][r][v];
                        }
#pragma unroll
                        for (int r = 0; r < RW; ++r)
#pragma unroll
                            for (int v = 0; v < V; ++v) ring[t][sj][r][v] = res[r][v];
                    } else {
                        store_cells(j, res);
                    }
                }
                advance();
            }
            return ok;
        };

        for (int ib = ib0; ib < iend; ib += P) {
            const bool fast = (ib - BT * R >= z0) && (ib + P - 1 - BT * R < z1) &&
                              (ib - BT * R >= R) && (ib + P - 1 - R < nz + R);
            bool ok;
            if (fast)
                ok = edge ? group(std::false_type{}, std::true_type{}, ib)
                          : group(std::false_type{}, std::false_type{}, ib);
            else
                ok = group(std::true_type{}, std::true_type{}, ib);
            if (!__syncthreads_and(ok)) {
                drain(ib);
                return;
            }
        }
    } else {
        // pa[t-1][p % P][r][v] = pending partial sum of level-t plane p, t = 1..bT
        Acc<MODE, C> pa[BT][P][RW][V];
#pragma unroll
        for (int t = 0; t < BT; ++t)
#pragma unroll
            for (int s = 0; s < P; ++s)
#pragma unroll
                for (int r = 0; r < RW; ++r)
#pragma unroll
                    for (int v = 0; v < V; ++v) pa[t][s][r][v].set(C(0));

        auto group = [&](auto check_tag, auto edge_tag, int ib) -> bool {
            constexpr bool CHECK = decltype(check_tag)::value;
            constexpr bool EDGE = decltype(edge_tag)::value;
            bool ok = true;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int i = ib + k;
                if (CHECK && i >= iend) return ok;
                if (CHECK) __syncthreads();  // iterations of halo planes may have no exchange
                C in[RW][V];
                load_plane(i, !CHECK || i < nplanes, in, ok);
#pragma unroll
                for (int t = 1; t <= BT; ++t) {
                    const int ar = i - (t - 1) * R;  // arriving level-(t-1) plane
                    C ext[RW + 2 * R][V];
                    exchange(in, ext);
                    C L[RW + 2 * R][R], Rt[RW + 2 * R][R];
#pragma unroll
                    for (int q = 0; q < RW + 2 * R; ++q) xshift(ext[q], L[q], Rt[q]);
#pragma unroll
                    for (int dz = -R; dz <= R; ++dz) {
                        const int b = ar - dz;  // pending level-t plane receiving its dz terms
                        const int sp = ((k - (t - 1) * R - dz) % P + P) % P;
                        if (CHECK && (b < R || b >= nz + R)) {
                            if (dz == 0 && t < BT) {
#pragma unroll
                                for (int r = 0; r < RW; ++r)
#pragma unroll
                                    for (int v = 0; v < V; ++v) pa[t - 1][sp][r][v].set(in[r][v]);
                            }
                            continue;
                        }
#pragma unroll
                        for (int r = 0; r < RW; ++r)
#pragma unroll
                            for (int dy = -R; dy <= R; ++dy)
#pragma unroll
                                for (int dx = -R; dx <= R; ++dx) {
                                    const int kk = ((dz + R) * P + (dy + R)) * P + (dx + R);
                                    const int q = R + r + dy;
#pragma unroll
                                    for (int v = 0; v < V; ++v) {
                                        const int s = v + dx;
                                        const C xv = s < 0 ? L[q][-s - 1] : (s >= V ? Rt[q][s - V] : ext[q][s]);
                                        if (dz == -R && dy == -R && dx == -R)
                                            pa[t - 1][sp][r][v].first(cf[kk], xv);
                                        else
                                            pa[t - 1][sp][r][v].add(cf[kk], xv);
                                    }
                                }
                    }
                    const int e = i - t * R;  // level-t plane completed now
                    const int se = ((k - t * R) % P + P) % P;
                    // a halo plane's pending value is its fixed copy: no per-step division
                    const bool inner = !CHECK || (e >= R && e < nz + R);
                    C out[RW][V];
#pragma unroll
                    for (int r = 0; r < RW; ++r)
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const C x = pa[t - 1][se][r][v].result();
                            out[r][v] = level_round<S>(inner ? post_op<POST>(x, a.post_c) : x);
                        }
                    if (t < BT) {
                        if (EDGE) {
                            int s = cs - t * R;  // plane e = i - t*R is t*R slots back
                            if (s < 0) s += D;
#pragma unroll
                            for (int r = 0; r < RW; ++r) {
                                const S *orig = cells_in_slot(e, s, r);
#pragma unroll
                                for (int v = 0; v < V; ++v)
                                    if (halo_bits & (1u << (r * V + v))) out[r][v] = load_c<S>(orig[v]);
                            }
                        }
#pragma unroll
                        for (int r = 0; r < RW; ++r)
#pragma unroll
                            for (int v = 0; v < V; ++v) in[r][v] = out[r][v];
                    } else if (!CHECK || (e >= z0 && e < z1)) {
                        store_cells(e, out);
                    }
                }
                advance();
            }
            return ok;
        };

        for (int ib = ib0; ib < iend; ib += P) {
            const bool fast = (ib - BT * R >= z0) && (ib + P - 1 - BT * R < z1) &&
                              (ib - BT * R >= R) && (ib + P - 1 + R < nz + R);
            bool ok;
            if (fast)
                ok = edge ? group(std::false_type{}, std::true_type{}, ib)
                          : group(std::false_type{}, std::false_type{}, ib);
            else
                ok = group(std::true_type{}, std::true_type{}, ib);
            if (!__syncthreads_and(ok)) {
                drain(ib);
                return;
            }
        }
    }
}

template <int SHAPE, int R, int BT, typename S, int MODE, int NW, int POST, int V_, int RW_>
cudaError_t launch_sweep3d(const PassDesc &d, cudaStream_t st)
{
    constexpr int N = NCoeff3<SHAPE, R>::value;
    using C = typename StorageTraits<S>::C;
    using G = Sweep3DGeom<S, SHAPE, BT, R, NW, V_, RW_>;
    // the descriptor must describe this kernel's tile (its TMA box too)
    if (d.tile_stride_x != G::TX - 2 * BT * R || d.tile_stride_y != G::TY - 2 * BT * R)
        return cudaErrorInvalidValue;
    Sweep3DArgs<S, N> a;
    a.dst = static_cast<S *>(d.dst);
    a.status = d.status;
    a.px = static_cast<int>(d.pitch);
    a.py = static_cast<int>(d.plane / d.pitch);
    a.nz = d.nz;
    a.ny = d.ny;
    a.nx = d.nx;
    a.tsx = d.tile_stride_x;
    a.tsy = d.tile_stride_y;
    a.xb0 = d.x_base;
    a.tiles_x = d.tiles_x;
    a.tiles_y = d.tiles_y;
    a.hsn = d.hsn;
    a.total_ctas = d.total_units;
    for (int k = 0; k < N; ++k) a.k.c[k] = static_cast<C>(d.coeffs[k]);
    a.post_c = static_cast<C>(d.post_c);
    auto fn = sweep3d_kernel<SHAPE, R, BT, S, MODE, NW, POST, V_, RW_>;
    if (G::SMEM_BYTES > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
    }
    fn<<<d.ctas, NW * 32, G::SMEM_BYTES, st>>>(d.tmap, a);
    return cudaGetLastError();
}

// PART_ = 1 registers the kernel as the narrow last-column kernel of the
// passes whose main kernel has the same key (same NW and RW: same tile rows).
// TILE_ > 0 registers it as a tile variant keyed by that width (the tuner
// times it beside the default tile of the same stencil and degree).
template <int SHAPE, int R, int BT, typename S, int MODE, int NW, int POST = POST_NONE,
          int V_ = CELLS_PER_LANE, int RW_ = 2, int PART_ = 0, int TILE_ = 0>
KernelEntry entry3d(int dtype)
{
    using G = Sweep3DGeom<S, SHAPE, BT, R, NW, V_, RW_>;
    static_assert(TILE_ == 0 || (TILE_ == G::TX && PART_ == 0), "a tile variant is keyed by its own width");
    KernelEntry e;
    e.key = KernelKey{3, SHAPE, R, dtype, BT, POST};
    e.key.part = PART_;
    e.key.tile = TILE_;
    e.launch = &launch_sweep3d<SHAPE, R, BT, S, MODE, NW, POST, V_, RW_>;
    e.func = reinterpret_cast<const void *>(&sweep3d_kernel<SHAPE, R, BT, S, MODE, NW, POST, V_, RW_>);
    e.threads = NW * 32;
    e.smem_bytes = G::SMEM_BYTES;
    e.tile_x = G::TX;
    e.tile_y = G::TY;
    e.units_per_cta = 1;
    return e;
}

}  // namespace an5d
