// sweep3d_box1.cuh -- one-level (bT = 1) 3D box sweep for radius 2..4 (sm_103a).
//
// Method: a high-order 3D box stencil has (2R+1)^3 terms per cell; the
// register cost of holding bT levels grows with that, so temporal blocking
// stops paying and the paper runs these stencils at bT = 1 (Table 5, box3d
// R2-R4; §6 on high-order stencils).  With one level there is no level
// exchange and no Dirichlet reset: each pass reads every input plane once
// (TMA) and writes the interior once.
//
// GB300 mapping (this library's design):
//  * a CTA of NW warps owns a tile of TY = RW*NW rows (y) by 128 cells (x),
//    streams z, and stores the (TY-2R) x (128-2R) interior of its tile;
//  * input planes are staged by TMA (every warp copies its own rows, one
//    1D row copy per lane) into a shared-memory ring of planes guarded by one
//    mbarrier per plane that all warps arrive on;
//    every thread reads its neighbours in y and x straight from the staged
//    plane (no shuffles, no exchange buffer);
//  * the 2R+1 output planes in flight are partial sums in registers
//    (Section 3.2, associative stencil optimisation): arriving plane p adds
//    its dz = p - b block of (dy, dx) terms to pending plane b, so every
//    output cell is the plain fma chain in canonical order (dz outer, then
//    dy, then dx); the completed plane is stored and the ring of partial
//    sums shifts by one (2R+1 x 8 register moves per plane, against
//    (2R+1)^3 x 8 fmas), which keeps the loop body a single copy.
#pragma once

#include "an5d_internal.h"
#include "device_common.cuh"
#include "sweep3d.cuh"

namespace an5d {

template <typename S, int R, int NW, int RW_> struct Box1Geom {
    static constexpr int V = CELLS_PER_LANE;
    static constexpr int RW = RW_;               // rows per warp
    static constexpr int TY = NW * RW;           // tile rows
    static constexpr int TX = 32 * V;            // tile columns
    static constexpr int P = 2 * R + 1;
    static constexpr int A = StorageTraits<S>::ALIGN_ELEMS;
    static constexpr int ROWBUF = TX + A;        // TMA box per row
    static constexpr int ROW_BYTES = ((ROWBUF * (int)sizeof(S) + 127) / 128) * 128;
    static constexpr int SLOT_BYTES = TY * ROW_BYTES;
    static constexpr int PF = PREFETCH_ROWS;     // planes in flight ahead
    // ring depth: the slot refilled at plane p held plane p - 2, which every
    // warp finished reading before the previous plane's CTA barrier
    static constexpr int D = PF + 2;
    // Lane 0 reads up to R cells left of its row's staged data: the ring
    // starts PAD bytes into the allocation so those reads stay inside it.
    // On the right, lane 31 reads up to A-1+R cells past the 128-cell tile,
    // which stays inside the 128-byte-rounded row.
    static constexpr int PAD = 128;
    static constexpr int SMEM_BYTES = PAD + D * SLOT_BYTES + D * 8 + 128;
    static_assert(SMEM_BYTES <= 232448, "shared memory per CTA exceeds 227 KB");
    static_assert(R * (int)sizeof(S) <= PAD, "left reads must stay in the pad");
    static_assert((A - 1 + TX + R) * (int)sizeof(S) <= ROW_BYTES, "right reads must stay in the row");
    static_assert(TX - 2 * R >= 8 && TY - 2 * R >= 2, "tile too small for R");
    static_assert(RW <= 32, "one TMA row per lane");
};

// E cells at p (shared memory) into w, with the widest reads the address
// allows: the row's misalignment is the same for every lane (a tile row keeps
// the global row's offset), so the choice does not diverge; 16-byte reads at
// a 16-byte lane stride take a quarter of the wavefronts of 4-byte reads.
template <typename S, int E> __device__ __forceinline__ void load_window(const S *p, typename StorageTraits<S>::C (&w)[E])
{
    const unsigned a = (unsigned)reinterpret_cast<uintptr_t>(p);
    if constexpr (std::is_same<S, float>::value && E % 4 == 0) {
        if ((a & 15u) == 0) {
#pragma unroll
            for (int i = 0; i < E / 4; ++i) {
                const float4 q = reinterpret_cast<const float4 *>(p)[i];
                w[4 * i] = q.x, w[4 * i + 1] = q.y, w[4 * i + 2] = q.z, w[4 * i + 3] = q.w;
            }
            return;
        }
    }
    if constexpr (std::is_same<S, float>::value && E % 2 == 0) {
        if ((a & 7u) == 0) {
#pragma unroll
            for (int i = 0; i < E / 2; ++i) {
                const float2 q = reinterpret_cast<const float2 *>(p)[i];
                w[2 * i] = q.x, w[2 * i + 1] = q.y;
            }
            return;
        }
    }
    if constexpr (std::is_same<S, double>::value && E % 2 == 0) {
        if ((a & 15u) == 0) {
#pragma unroll
            for (int i = 0; i < E / 2; ++i) {
                const double2 q = reinterpret_cast<const double2 *>(p)[i];
                w[2 * i] = q.x, w[2 * i + 1] = q.y;
            }
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) w[e] = load_c<S>(p[e]);
}

template <int R, typename S, int NW, int RW_>
__global__ void __launch_bounds__(NW * 32, 1)
    box1_kernel(const __grid_constant__ CUtensorMap tmap,
                const Sweep3DArgs<S, NCoeff3<SH_BOX, R>::value> a)
{
    using C = typename StorageTraits<S>::C;
    using G = Box1Geom<S, R, NW, RW_>;
    constexpr int V = G::V, RW = G::RW, TY = G::TY, P = G::P, D = G::D, A = G::A, PF = G::PF;
    constexpr int NQ = RW + 2 * R;  // input rows a warp reads
    extern __shared__ __align__(128) unsigned char smem[];

    const int cta = blockIdx.x;
    if (cta >= a.total_ctas) return;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    // ---- tile geometry (one level: the tile starts R cells before its interior) ----
    const int xt = cta % a.tiles_x;
    const int yt = (cta / a.tiles_x) % a.tiles_y;
    const int zb = cta / (a.tiles_x * a.tiles_y);
    const int x0 = xt * a.tsx;                // padded column of the tile's first cell
    const int yb = yt * a.tsy;                // padded row of the tile's first row
    const int px = a.px, py = a.py, nx = a.nx, ny = a.ny, nz = a.nz;
    const int z0 = R + zb * a.hsn;
    const int z1 = min(z0 + a.hsn, nz + R);
    const int pbeg = z0 - R, pend = z1 + R;   // input planes [pbeg, pend)
    const long plane = (long)px * py;

    const int col0 = x0 + lane * V;
    const int row0 = yb + warp * RW;
    const int sc0 = max(R, x0 + R), sc1 = min(nx + R, x0 + R + a.tsx);
    const int sr0 = max(R, yb + R), sr1 = min(ny + R, yb + R + a.tsy);
    unsigned store_bits = 0;                  // bit r*V+v
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int y = row0 + r, x = col0 + v;
            if (y >= sr0 && y < sr1 && x >= sc0 && x < sc1) store_bits |= 1u << (r * V + v);
        }

    // aligned by pointer arithmetic on the shared array, so that the compiler
    // keeps the window reads below in the shared address space
    unsigned char *const base = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    unsigned char *const ring = base + G::PAD;
    uint64_t *const bars = reinterpret_cast<uint64_t *>(ring + D * G::SLOT_BYTES);
    int *const status = a.status;

    // TMA of the tile rows of plane p into ring slot s: every warp copies its
    // own RW rows (lane r copies row warp*RW + r) and arrives on the slot's
    // mbarrier with their byte count; the plane is complete when all NW
    // warps arrived and every row landed.
    auto issue_plane = [&](int p, int s) {
        if (lane == 0) mbar_expect_tx(&bars[s], RW * G::ROWBUF * (int)sizeof(S));
        __syncwarp();
        if (lane < RW) {
            const int row = warp * RW + lane;
            const long lin = (long)p * plane + (long)(yb + row) * px + x0;
            fence_proxy_async();
            tma_load_1d(ring + s * G::SLOT_BYTES + row * G::ROW_BYTES, &tmap,
                        (int)(lin & ~long(A - 1)), &bars[s]);
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < D; ++s) mbar_init(&bars[s], NW);
        fence_mbar_init();
    }
    __syncthreads();
    for (int q = 0; q < PF; ++q)
        if (pbeg + q < pend) issue_plane(pbeg + q, q);

    // acc[d][r][v]: pending output plane p - R + d (it next receives the
    // dz = R - d block of plane p); acc[0] completes with plane p.
    Acc<MODE_PLAIN, C> acc[P][RW][V];
#pragma unroll
    for (int d = 0; d < P; ++d)
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[d][r][v].set(C(0));

    const auto &cf = a.k.c;
    S *const dst = a.dst;
    int cs = 0;
    uint32_t cpar = 0;
    for (int p = pbeg; p < pend; ++p) {
        if (p + PF < pend) {
            int s = cs + PF;
            if (s >= D) s -= D;
            issue_plane(p + PF, s);
        }
        const bool ok = mbar_wait_warp(&bars[cs], cpar, status);
        if (!__syncthreads_and(ok)) {
            // the warps that gave up wait (bounded) for the copies still in flight
            // (every warp's rows of planes p .. p+PF land on these mbarriers)
            if (!ok) {
                int s = cs;
                uint32_t ph = cpar;
                for (int q = p; q <= p + PF && q < pend; ++q) {
                    if (!mbar_wait_warp(&bars[s], ph, status)) break;
                    if (++s == D) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            return;
        }
        const long pl = (long)p * plane;
        const unsigned char *slot = ring + cs * G::SLOT_BYTES;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            // tile row warp*RW - R + q, clamped into the tile: clamped rows only
            // feed cells outside the stored interior
            int tr = warp * RW - R + q;
            tr = tr < 0 ? 0 : (tr >= TY ? TY - 1 : tr);
            const int off = (int)((pl + (long)(yb + tr) * px + x0) & long(A - 1));
            const S *src = reinterpret_cast<const S *>(slot + tr * G::ROW_BYTES) + off + lane * V - R;
            C w[V + 2 * R];  // cells x-R .. x+V-1+R of this row
            load_window<S, V + 2 * R>(src, w);
#pragma unroll
            for (int d = 0; d < P; ++d) {
                const int dz = R - d;
#pragma unroll
                for (int r = 0; r < RW; ++r) {
                    const int dy = q - R - r;
                    if (dy < -R || dy > R) continue;
#pragma unroll
                    for (int dx = -R; dx <= R; ++dx) {
                        const int kk = ((dz + R) * P + (dy + R)) * P + (dx + R);
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            if (dz == -R && dy == -R && dx == -R)
                                acc[d][r][v].first(cf[kk], w[v + dx + R]);
                            else
                                acc[d][r][v].add(cf[kk], w[v + dx + R]);
                        }
                    }
                }
            }
        }
        // output plane p - R is complete
        const int b = p - R;
        if (b >= z0) {
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                S *out = dst + (b * plane + (long)(row0 + r) * px + col0);
#pragma unroll
                for (int v = 0; v < V; ++v)
                    st_pred<S>(out + v, to_storage<S>(acc[0][r][v].result()), store_bits, r * V + v);
            }
        }
#pragma unroll
        for (int d = 0; d + 1 < P; ++d)
#pragma unroll
            for (int r = 0; r < RW; ++r)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[d][r][v] = acc[d + 1][r][v];
        if (++cs == D) {
            cs = 0;
            cpar ^= 1u;
        }
    }
}

template <int R, typename S, int NW, int RW_>
cudaError_t launch_box1(const PassDesc &d, cudaStream_t st)
{
    constexpr int N = NCoeff3<SH_BOX, R>::value;
    using C = typename StorageTraits<S>::C;
    using G = Box1Geom<S, R, NW, RW_>;
    // the descriptor must describe this kernel's tile (one level: bT = 1)
    if (d.tile_stride_x != G::TX - 2 * R || d.tile_stride_y != G::TY - 2 * R) return cudaErrorInvalidValue;
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
    a.xb0 = d.x_base;  // unused: one-level tiles start at column 0
    a.tiles_x = d.tiles_x;
    a.tiles_y = d.tiles_y;
    a.hsn = d.hsn;
    a.total_ctas = d.total_units;
    for (int k = 0; k < N; ++k) a.k.c[k] = static_cast<C>(d.coeffs[k]);
    a.post_c = C(0);
    auto fn = box1_kernel<R, S, NW, RW_>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    fn<<<d.ctas, NW * 32, G::SMEM_BYTES, st>>>(d.tmap, a);
    return cudaGetLastError();
}

template <int R, typename S, int NW, int RW_>
KernelEntry entry_box1(int dtype)
{
    using G = Box1Geom<S, R, NW, RW_>;
    KernelEntry e;
    e.key = KernelKey{3, SH_BOX, R, dtype, 1};
    e.launch = &launch_box1<R, S, NW, RW_>;
    e.func = reinterpret_cast<const void *>(&box1_kernel<R, S, NW, RW_>);
    e.threads = NW * 32;
    e.smem_bytes = G::SMEM_BYTES;
    e.tile_x = G::TX;
    e.tile_y = G::TY;
    e.units_per_cta = 1;
    return e;
}

}  // namespace an5d
