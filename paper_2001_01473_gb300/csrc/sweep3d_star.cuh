// sweep3d_star.cuh -- 2.5D-blocked, temporally blocked FP32 3D star sweep
// with one CTA barrier per streamed plane (sm_103a).
//
// Method (AN5D, Section 3.1, Fig. 1; Section 3.2): tile y and x, stream z,
// fuse bT time levels per pass; level t lags level t-1 by R planes and its
// valid region shrinks by R cells per side in y and x; only level bT's
// compute region is stored; z is cut into stream blocks of hsn planes.
//
// GB300 mapping (this library's design):
//  * a CTA of NW warps owns TY = RW*NW rows (y) by TX = 32*V cells (x); each
//    warp owns RW rows, each lane V consecutive x cells of them;
//  * input planes are staged by TMA into a shared-memory ring, one elected
//    lane per warp copying that warp's rows and the warp waiting on its own
//    mbarrier (no CTA-wide synchronisation on the ring);
//  * each level keeps the 2R+1 most recent planes of the thread's cells in a
//    fixed register ring indexed by plane mod (2R+1) (Section 3.2 register
//    allocation): these are the z neighbours;
//  * x neighbours travel by warp shuffles;
//  * y neighbours: level t's plane j is needed by level t+1 only R planes
//    later (level t+1 lags by R), so every level publishes each new plane to
//    a shared-memory buffer of R+1 plane slots, and level t+1 reads its y
//    neighbours there R iterations after.  One CTA barrier per streamed plane
//    then orders every publication before every read, whatever bT is (the
//    paper's double-buffered shared memory, Section 3.2, with one barrier per
//    plane instead of one per level);
//  * the chain is the scalar fma chain in the canonical order with the
//    coefficients as constant-bank operands (a packed f32x2 chain measured
//    slower here: repacking the odd x shifts and loading the packed
//    coefficients cost more issue slots than the pairs save);
//  * shared-memory offsets are computed once per thread and advanced per
//    plane, so the per-plane bookkeeping is a few integer adds;
//  * tiles start on even columns (the host aligns the tile origin), so with
//    an even row pitch every staged row of a lane starts on an 8-byte
//    boundary: it is read as one 16-byte vector or two 8-byte pairs;
//  * Dirichlet halo: halo planes are copied level to level; in tiles that
//    touch the domain boundary, halo cells are reset to their input values
//    after every level (Section 3.1).
#pragma once

#include <type_traits>

#include "sweep3d.cuh"

namespace an5d {

__device__ __forceinline__ void mbar_init_u32(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx_u32(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_u32(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Warp-uniform bounded wait (same contract as mbar_wait_warp).
__device__ __forceinline__ bool mbar_wait_warp_u32(uint32_t bar, uint32_t parity, int *status)
{
    if (__all_sync(FULL_MASK, mbar_try_wait_u32(bar, parity))) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (__all_sync(FULL_MASK, mbar_try_wait_u32(bar, parity))) return true;
        const bool late = (global_ns() - t0) > WAIT_LIMIT_NS;
        if (__any_sync(FULL_MASK, late)) {
            if ((threadIdx.x & 31) == 0) atomicOr(status, STATUS_TIMEOUT);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_1d_u32(uint32_t dst, const CUtensorMap *map, int32_t x, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2}], [%3];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(bar)
        : "memory");
}

template <int BT, int R, int NW, int V_, int RW_> struct Star3DGeom {
    static constexpr int V = V_;
    static constexpr int RW = RW_;
    static constexpr int TY = NW * RW;
    static constexpr int TX = 32 * V;
    static constexpr int P = 2 * R + 1;
    static constexpr int A = 4;                                             // 16 bytes of FP32
    static constexpr int ROWBUF = TX + A;                                   // TMA box per row
    static constexpr int ROW_BYTES = ((ROWBUF * 4 + 127) / 128) * 128;
    static constexpr int SLOT_BYTES = TY * ROW_BYTES;
    // published planes of levels 0..BT-1: R+1 slots each, R pad rows above and
    // below the tile (they feed only cells outside the valid region)
    static constexpr int XROWS = TY + 2 * R;
    static constexpr int XSLOT_B = XROWS * TX * 4;
    static constexpr int XLEVEL_B = (R + 1) * XSLOT_B;
    static constexpr int XB_BYTES = BT * XLEVEL_B;
    static constexpr int PF_FIT = (232448 - 128 - XB_BYTES) / (SLOT_BYTES + NW * 8) - 1;
    static constexpr int PF = PF_FIT > 6 ? 6 : PF_FIT;                     // planes in flight ahead
    static constexpr int D = PF + 1;                                        // staging ring depth
    static constexpr int SMEM_BYTES = D * SLOT_BYTES + XB_BYTES + D * NW * 8 + 128;
    static_assert(PF >= 2, "shared memory too small for the staging ring");
    static_assert(SMEM_BYTES <= 232448, "shared memory per CTA exceeds 227 KB");
    static_assert(TX - 2 * BT * R >= 8 && TY - 2 * BT * R >= 2, "tile too small for bT*R");
    static_assert(R <= V, "radius must not exceed cells per lane");
    static_assert(RW * V <= 32, "cell bit masks");
    static_assert(V == 1 || V == 2 || V == 4, "published rows move as 4-, 8- or 16-byte vectors");
};

template <int R, int BT, int NW, int V_, int RW_>
__global__ void __launch_bounds__(NW * 32, 1)
    star3d_kernel(const __grid_constant__ CUtensorMap tmap, const Sweep3DArgs<float, NCoeff3<SH_STAR, R>::value> a)
{
    using G = Star3DGeom<BT, R, NW, V_, RW_>;
    constexpr int V = G::V, RW = G::RW, TX = G::TX, P = G::P, D = G::D, PF = G::PF;
    constexpr int ROW_BYTES = G::ROW_BYTES, SLOT_BYTES = G::SLOT_BYTES;
    constexpr int XSLOT_B = G::XSLOT_B, XLEVEL_B = G::XLEVEL_B;
    extern __shared__ __align__(128) unsigned char smem[];

    const int cta = blockIdx.x;
    if (cta >= a.total_ctas) return;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    // ---- tile geometry ----
    const int xt = cta % a.tiles_x;
    const int yt = (cta / a.tiles_x) % a.tiles_y;
    const int zb = cta / (a.tiles_x * a.tiles_y);
    const int x0 = a.xb0 - BT * R + xt * a.tsx;  // padded column of the tile's first cell
    const int yb = R - BT * R + yt * a.tsy;      // padded row of the tile's first row
    const int px = a.px, nz = a.nz, ny = a.ny, nx = a.nx;
    const int pstride = a.py * px;                // elements per padded plane
    const int nplanes = nz + 2 * R;
    const int z0 = R + zb * a.hsn;
    const int z1 = min(z0 + a.hsn, nz + R);
    const int zs = max(0, z0 - BT * R);
    const int ib0 = zs - zs % P;
    const int iend = z1 + BT * R;
    const int pend = min(nplanes, iend);           // planes requested: exactly the planes consumed

    const int col0 = x0 + lane * V;
    const int row0 = yb + warp * RW;
    const int sc0 = max(R, x0 + BT * R), sc1 = min(nx + R, x0 + BT * R + a.tsx);
    const int sr0 = max(R, yb + BT * R), sr1 = min(ny + R, yb + BT * R + a.tsy);
    unsigned halo_bits = 0, store_bits = 0;  // bit r*V+v
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int y = row0 + r, x = col0 + v;
            if (y < R || y >= ny + R || x < R || x >= nx + R) halo_bits |= 1u << (r * V + v);
            if (y >= sr0 && y < sr1 && x >= sc0 && x < sc1) store_bits |= 1u << (r * V + v);
        }
    const bool edge = __syncthreads_or(halo_bits != 0) != 0;
    // every staged row of this tile starts on an 8-byte boundary (cells as pairs)
    const bool even = ((x0 | px) & 1) == 0;

    // ---- shared memory (32-bit addresses) ----
    const uint32_t base = (smem_u32(smem) + 127u) & ~127u;
    // The same memory as a pointer derived from the shared array, for the
    // published planes and the staged rows: the compiler then knows these are
    // shared-memory accesses and may schedule them freely between barriers.
    unsigned char *const smb = smem + (base - smem_u32(smem));
    auto SF = [&](uint32_t a) -> float * { return reinterpret_cast<float *>(smb + (a - base)); };
    const uint32_t stage = base;
    const uint32_t xbuf = base + D * SLOT_BYTES;
    const uint32_t bars = xbuf + G::XB_BYTES;
    const uint32_t my_bar0 = bars + warp * 8;                       // slot s: + s * NW * 8
    const uint32_t my_stage0 = stage + warp * RW * ROW_BYTES + lane * V * 4;
    const uint32_t my_xb = xbuf + ((R + warp * RW) * TX + lane * V) * 4;  // level 0, slot 0, own row 0
    int *const status = a.status;
    // padded linear index of this warp's row 0 of plane 0 at the tile's first cell
    const int rl0 = row0 * px + x0;
    const int rmis = px & 3;                  // misalignment step from one row to the next

    // ---- staging: one elected lane copies the warp's RW rows of each plane ----
    int nissue = ib0;  // next plane this warp requests
    auto issue_plane = [&](int p, int s) {
        // No proxy fence: the slot's previous rows were read by this warp only
        // (other warps read published copies), iterations before the refill.
        if (lane == 0) {
            const uint32_t bar = my_bar0 + s * NW * 8;
            mbar_expect_tx_u32(bar, RW * G::ROWBUF * 4);
            const int lin = p * pstride + rl0;
#pragma unroll
            for (int r = 0; r < RW; ++r)
                tma_load_1d_u32(stage + s * SLOT_BYTES + (warp * RW + r) * ROW_BYTES, &tmap,
                                (lin + r * px) & ~3, bar);
        }
        nissue = p + 1;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < D * NW; ++s) mbar_init_u32(bars + 8 * s, 1);
        fence_mbar_init();
    }
    __syncthreads();
    for (int q = 0; q < PF; ++q)
        if (ib0 + q < pend) issue_plane(ib0 + q, q);

    int cs = 0, cur_p = ib0;   // ring slot and phase of plane cur_p
    uint32_t cpar = 0;
    int fpl = -1, fcs = 0;     // first plane whose wait gave up (-1: none), its slot and phase
    uint32_t fpar = 0;
    int pmis = (ib0 * pstride + rl0) & 3;  // misalignment of this warp's row 0 of plane cur_p
    const int pmis_step = pstride & 3;
    // byte offsets of the published slots written (plane i) and read (plane
    // i - R) in iteration i: slot i mod (R+1) and (i+1) mod (R+1)
    int wofs = (ib0 % (R + 1)) * XSLOT_B;
    int rofs = wofs + XSLOT_B == (R + 1) * XSLOT_B ? 0 : wofs + XSLOT_B;

    const auto &cf = a.k.c;
    float *const dst = a.dst;

    // Iteration i: request plane i+PF (its slot last held plane i-1, read by
    // this warp already), wait for plane i and copy this thread's cells to
    // registers.  After a wait gives up the warp stops requesting planes and
    // computes on zeros, so that every CTA barrier is still reached.
    auto load_plane = [&](bool pairs, int i, bool have, float (&cell)[RW][V], bool &ok) {
        if (ok && i + PF < pend) {
            int s = cs + PF;
            if (s >= D) s -= D;
            issue_plane(i + PF, s);
        }
        if (have && ok) {
            ok = mbar_wait_warp_u32(my_bar0 + cs * NW * 8, cpar, status);
            if (!ok) {
                fpl = i;
                fcs = cs;
                fpar = cpar;
            }
        }
        if (have && ok) {
            const uint32_t src = my_stage0 + cs * SLOT_BYTES;
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const int mis = (pmis + r * rmis) & 3;
                const float *qp = SF(src + r * ROW_BYTES + mis * 4);
                bool done = false;
                if constexpr (V == 4) {
                    if (mis == 0) {  // a 16-byte aligned row: one vector
                        const float4 f = *reinterpret_cast<const float4 *>(qp);
                        cell[r][0] = f.x, cell[r][1] = f.y, cell[r][2] = f.z, cell[r][3] = f.w;
                        done = true;
                    }
                }
                if (done) {
                } else if (pairs && V % 2 == 0) {
#pragma unroll
                    for (int h = 0; h < V / 2; ++h) {
                        const float2 f = reinterpret_cast<const float2 *>(qp)[h];
                        cell[r][2 * h] = f.x, cell[r][2 * h + 1] = f.y;
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) cell[r][v] = qp[v];
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < RW; ++r)
#pragma unroll
                for (int v = 0; v < V; ++v) cell[r][v] = 0.f;
        }
    };
    auto advance = [&]() {
        ++cur_p;
        pmis = (pmis + pmis_step) & 3;
        if (++cs == D) {
            cs = 0;
            cpar ^= 1u;
        }
        wofs = rofs;
        rofs = rofs + XSLOT_B == (R + 1) * XSLOT_B ? 0 : rofs + XSLOT_B;
    };
    // After a timeout anywhere in the CTA every warp leaves; first it waits
    // (bounded) for its own copies still in flight.
    auto drain = [&]() {
        int p0 = cur_p, s = cs;
        uint32_t ph = cpar;
        if (fpl >= 0) p0 = fpl, s = fcs, ph = fpar;
        for (int p = p0; p < nissue; ++p) {
            if (!mbar_wait_warp_u32(my_bar0 + s * NW * 8, ph, status)) break;
            if (++s == D) {
                s = 0;
                ph ^= 1u;
            }
        }
    };
    // Publish level t's newest plane: the rows of this warp that other warps
    // read (the R rows at each end of the warp's RW rows).
    auto publish = [&](int t, const float (&w)[RW][V]) {
        const uint32_t p = my_xb + t * XLEVEL_B + wofs;
#pragma unroll
        for (int r = 0; r < RW; ++r)
            if (r < R || r >= RW - R) {
                float *q = SF(p + r * TX * 4);
                if constexpr (V == 4) *reinterpret_cast<float4 *>(q) = make_float4(w[r][0], w[r][1], w[r][2], w[r][3]);
                else if constexpr (V == 2) *reinterpret_cast<float2 *>(q) = make_float2(w[r][0], w[r][1]);
                else q[0] = w[r][0];
            }
    };
    auto store_cells = [&](int j, const float (&w)[RW][V]) {
        float *out = dst + ((size_t)j * pstride + (size_t)row0 * px + col0);
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (store_bits & (1u << (r * V + v))) out[r * px + v] = w[r][v];
    };

    // ring[t][p % P][r][v] = level-t plane p at this thread's cells, t = 0..bT-1
    float ring[BT][P][RW][V];
#pragma unroll
    for (int t = 0; t < BT; ++t)
#pragma unroll
        for (int s = 0; s < P; ++s)
#pragma unroll
            for (int r = 0; r < RW; ++r)
#pragma unroll
                for (int v = 0; v < V; ++v) ring[t][s][r][v] = 0.f;

    auto group = [&](auto check_tag, auto edge_tag, auto pairs_tag, int ib) -> bool {
        constexpr bool CHECK = decltype(check_tag)::value;
        constexpr bool EDGE = decltype(edge_tag)::value;
        constexpr bool PAIRS = decltype(pairs_tag)::value;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const int i = ib + k;
            if (CHECK && i >= iend) return ok;
            load_plane(PAIRS, i, !CHECK || i < nplanes, ring[0][k], ok);
            publish(0, ring[0][k]);
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
                // y neighbours of level t-1's plane j from other warps, published
                // R iterations ago (tile row warp*RW + q at nb + q*TX*4)
                const uint32_t nb = my_xb + (t - 1) * XLEVEL_B + rofs;
                float res[RW][V];
#pragma unroll
                for (int r = 0; r < RW; ++r) {
                    float x[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) x[v] = ring[t - 1][sj][r][v];
                    float L[R], Rt[R];
#pragma unroll
                    for (int d = 1; d <= R; ++d) {
                        L[d - 1] = __shfl_up_sync(FULL_MASK, x[V - d], 1);
                        Rt[d - 1] = __shfl_down_sync(FULL_MASK, x[d - 1], 1);
                    }
                    float acc[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[v] = __fmul_rn(cf[0], x[v]);
                    int kk = 1;
#pragma unroll
                    for (int ii = -R; ii <= R; ++ii) {
                        if (ii == 0) continue;
#pragma unroll
                        for (int v = 0; v < V; ++v) {  // dx = ii
                            const int s = v + ii;
                            acc[v] = __fmaf_rn(cf[kk], s < 0 ? L[-s - 1] : (s >= V ? Rt[s - V] : x[s]), acc[v]);
                        }
                        const int q = r + ii;  // dy = ii
                        if (q >= 0 && q < RW) {
#pragma unroll
                            for (int v = 0; v < V; ++v) acc[v] = __fmaf_rn(cf[kk + 1], ring[t - 1][sj][q][v], acc[v]);
                        } else {
                            float y[V];
                            const float *yp = SF(nb + q * TX * 4);
                            if constexpr (V == 4) {
                                const float4 f = *reinterpret_cast<const float4 *>(yp);
                                y[0] = f.x, y[1] = f.y, y[2] = f.z, y[3] = f.w;
                            } else if constexpr (V == 2) {
                                const float2 f = *reinterpret_cast<const float2 *>(yp);
                                y[0] = f.x, y[1] = f.y;
                            } else {
                                y[0] = yp[0];
                            }
#pragma unroll
                            for (int v = 0; v < V; ++v) acc[v] = __fmaf_rn(cf[kk + 1], y[v], acc[v]);
                        }
                        const int sz = ((k - t * R + ii) % P + P) % P;  // dz = ii
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = __fmaf_rn(cf[kk + 2], ring[t - 1][sz][r][v], acc[v]);
                        kk += 3;
                    }
#pragma unroll
                    for (int v = 0; v < V; ++v) res[r][v] = acc[v];
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
                    publish(t, res);
                } else {
                    store_cells(j, res);
                }
            }
            advance();
            if (k < P - 1) __syncthreads();  // publications of iteration i before reads of i + 1
        }
        return ok;
    };

    using T_ = std::true_type;
    using F_ = std::false_type;
    for (int ib = ib0; ib < iend; ib += P) {
        const bool fast = (ib - BT * R >= z0) && (ib + P - 1 - BT * R < z1) &&
                          (ib - BT * R >= R) && (ib + P - 1 - R < nz + R);
        bool ok;
        if (fast && !edge && even)
            ok = group(F_{}, F_{}, T_{}, ib);
        else if (fast)
            ok = group(F_{}, T_{}, F_{}, ib);
        else
            ok = group(T_{}, T_{}, F_{}, ib);
        if (!__syncthreads_and(ok)) {
            drain();
            return;
        }
    }
}

template <int R, int BT, int NW, int V_, int RW_>
cudaError_t launch_star3d(const PassDesc &d, cudaStream_t st)
{
    constexpr int N = NCoeff3<SH_STAR, R>::value;
    using G = Star3DGeom<BT, R, NW, V_, RW_>;
    // the descriptor must describe this kernel's tile (its TMA box too)
    if (d.tile_stride_x != G::TX - 2 * BT * R || d.tile_stride_y != G::TY - 2 * BT * R)
        return cudaErrorInvalidValue;
    Sweep3DArgs<float, N> a;
    a.dst = static_cast<float *>(d.dst);
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
    for (int k = 0; k < N; ++k) a.k.c[k] = static_cast<float>(d.coeffs[k]);
    a.post_c = 0.f;
    auto fn = star3d_kernel<R, BT, NW, V_, RW_>;
    if (G::SMEM_BYTES > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
    }
    fn<<<d.ctas, NW * 32, G::SMEM_BYTES, st>>>(d.tmap, a);
    return cudaGetLastError();
}

// PART_ = 1 registers the kernel as the narrow last-column kernel of the
// passes whose main kernel has the same key (same NW and RW: same tile rows);
// with PART_ = 0 and another cells-per-lane count than the default, the
// kernel is a tile variant of its width.
template <int R, int BT, int NW, int V_ = CELLS_PER_LANE, int RW_ = 2, int PART_ = 0>
KernelEntry entry_star3d()
{
    using G = Star3DGeom<BT, R, NW, V_, RW_>;
    KernelEntry e;
    e.key = KernelKey{3, SH_STAR, R, DT_F32, BT, POST_NONE};
    e.key.part = PART_;
    // a main kernel of another width is a tile variant, keyed by its width
    if (PART_ == 0 && V_ != CELLS_PER_LANE) e.key.tile = G::TX;
    e.launch = &launch_star3d<R, BT, NW, V_, RW_>;
    e.func = reinterpret_cast<const void *>(&star3d_kernel<R, BT, NW, V_, RW_>);
    e.threads = NW * 32;
    e.smem_bytes = G::SMEM_BYTES;
    e.tile_x = G::TX;
    e.tile_y = G::TY;
    e.units_per_cta = 1;
    return e;
}

}  // namespace an5d
