// batch.cu -- batched form: many independent 2D grids of uneven size, shape,
// radius and length advanced in one persistent launch, replayed as a CUDA
// graph.  (No counterpart in the paper, whose host code runs one grid at a
// time; the per-tile work is the same N.5D-blocked warp tile as the
// single-grid sweep.)
//
// Work items are (grid, x tile, stream block, pass), enumerated pass-major
// over all grids.  A warp takes the next item from a global counter, waits
// until the item's 3x3 neighbourhood of tiles has finished the previous pass
// (their outputs are its inputs, and their reads of its output buffer are
// over), runs the pass, and publishes its own pass counter.  Every item waits
// only on items enumerated before it, which resident warps already hold, so
// the queue cannot deadlock; every wait is bounded and gives up with an
// error status instead of hanging.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "an5d.h"
#include "an5d_internal.h"
#include "sweep2d.cuh"

namespace an5d {

// Stencil classes of the batched form and the degrees built for each.
constexpr int BATCH_CLASSES = 4;  // star R1, star R2, box R1, box R2
constexpr int BATCH_MENU = 3;
__host__ __device__ constexpr int batch_menu(int cls, int i)
{
    // radius 1: bT 1, 4, 8; radius 2: bT 1, 2, 4 (degree 1 also runs remainders)
    return (cls % 2 == 0) ? (i == 0 ? 1 : (i == 1 ? 4 : 8)) : (i == 0 ? 1 : (i == 1 ? 2 : 4));
}
// A wider tile (6 cells per lane, 192 cells) is built for one degree per
// class (radius 1: bT 4, radius 2: bT 2) and for its remainder degree 1:
// the level rings of the larger degrees would not fit the kernel's registers.
__host__ __device__ constexpr int batch_wide_deg(int cls) { return (cls % 2 == 0) ? 4 : 2; }
constexpr int BATCH_WIDE_V = 6;
constexpr int BATCH_MAX_N = 25;
constexpr int BATCH_WARPS = 4;

struct alignas(64) BatchGrid {
    CUtensorMap map[3];   // 1D maps over in, out, scratch
    float *buf[3];        // in (never written), out, scratch
    int pitch, ny, nx, radius, cls;
    int bt, full, rem, passes;  // degree, full-degree passes, remainder passes, total
    int rdeg[8];                // degrees of the remainder passes (T mod bT split over the menu)
    int lead;                   // bT*R: tiles start this far left of their compute region
    int v;                      // cells per lane of the grid's tiles (4 or 6)
    int stride, tiles_x, hsn, nsb;
    int counter_base;
    float coeffs[BATCH_MAX_N];
};

struct BatchItem {
    int g, xt, sb, pass;
};

// Shared memory per warp: the largest ring among the built instantiations.
template <int SHAPE, int R, int BT, int V = CELLS_PER_LANE> constexpr int batch_ring_bytes()
{
    return Sweep2DGeom<float, BT, R, V>::WARP_BYTES;
}
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int BATCH_WARP_BYTES =
    cmax(cmax(cmax(batch_ring_bytes<SH_BOX, 1, 8>(), batch_ring_bytes<SH_BOX, 2, 4>()),
              cmax(batch_ring_bytes<SH_STAR, 1, 8>(), batch_ring_bytes<SH_STAR, 2, 4>())),
         cmax(cmax(batch_ring_bytes<SH_BOX, 1, 4, BATCH_WIDE_V>(), batch_ring_bytes<SH_BOX, 2, 2, BATCH_WIDE_V>()),
              cmax(batch_ring_bytes<SH_STAR, 1, 4, BATCH_WIDE_V>(), batch_ring_bytes<SH_STAR, 2, 2, BATCH_WIDE_V>())));
constexpr int BATCH_SMEM = BATCH_WARPS * BATCH_WARP_BYTES + 128;

struct Coeffs25 {
    float c[BATCH_MAX_N];
};

// One pass of one tile with a given stencil and degree; invalidates the
// ring's mbarriers afterwards so that the next item can initialise its own.
template <int SHAPE, int R, int BT, int V = CELLS_PER_LANE>
__device__ __noinline__ bool batch_tile(const Tile2D tg, const CUtensorMap *map, float *dst, int *status,
                                        unsigned char *ring, const float *gc)
{
    constexpr int N = NCoeff2<SHAPE, R>::value;
    Coeffs25 cf;
#pragma unroll
    for (int k = 0; k < N; ++k) cf.c[k] = gc[k];
    const bool ok = sweep2d_tile<SHAPE, R, BT, float, MODE_PLAIN, false, decltype(cf.c), decltype(cf.c), false, true,
                                 POST_NONE, V>(tg, map, dst, status, ring, cf.c, cf.c);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        using G = Sweep2DGeom<float, BT, R, V>;
        uint64_t *bars = reinterpret_cast<uint64_t *>(ring + G::D * G::SLOT_BYTES);
        for (int s = 0; s < G::D; ++s)
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bars[s])) : "memory");
    }
    __syncwarp();
    return ok;
}

template <int SHAPE, int R>
__device__ __forceinline__ bool batch_dispatch_deg(int deg, int v, const Tile2D &tg, const CUtensorMap *map,
                                                   float *dst, int *status, unsigned char *ring, const float *gc)
{
    constexpr int cls = (SHAPE == SH_STAR ? 0 : 2) + (R - 1);
    if (v == BATCH_WIDE_V) {
        if (deg == batch_wide_deg(cls))
            return batch_tile<SHAPE, R, batch_wide_deg(cls), BATCH_WIDE_V>(tg, map, dst, status, ring, gc);
        return batch_tile<SHAPE, R, 1, BATCH_WIDE_V>(tg, map, dst, status, ring, gc);
    }
    if (deg == batch_menu(cls, 1)) return batch_tile<SHAPE, R, batch_menu(cls, 1)>(tg, map, dst, status, ring, gc);
    if (deg == batch_menu(cls, 2)) return batch_tile<SHAPE, R, batch_menu(cls, 2)>(tg, map, dst, status, ring, gc);
    return batch_tile<SHAPE, R, 1>(tg, map, dst, status, ring, gc);
}

__global__ void __launch_bounds__(BATCH_WARPS * 32)
    batch_kernel(const BatchGrid *__restrict__ grids, const BatchItem *__restrict__ items, int n_items,
                 int *queue, int *counters, int *status, int *abort_flag, int stall_item)
{
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *const base = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char *const ring = base + warp * BATCH_WARP_BYTES;
    while (true) {
        int it = 0;
        if (lane == 0) it = atomicAdd(queue, 1);
        it = __shfl_sync(FULL_MASK, it, 0);
        if (it >= n_items) break;
        if (__shfl_sync(FULL_MASK, lane == 0 ? *(volatile int *)abort_flag : 0, 0)) break;
        const BatchItem w = items[it];
        const BatchGrid &g = grids[w.g];
        // wait until the 3x3 neighbourhood has completed pass w.pass - 1
        bool ok = true;
        int need = w.pass;
        if (stall_item == it) need = 1 << 30;  // fault injection (tests only): never satisfied
        if (need > 0 && lane < 9) {
            const int xt = w.xt + lane % 3 - 1, sb = w.sb + lane / 3 - 1;
            if (xt >= 0 && xt < g.tiles_x && sb >= 0 && sb < g.nsb) {
                const int *c = counters + g.counter_base + sb * g.tiles_x + xt;
                if (ld_acquire(c) < need) {
                    const uint64_t t0 = global_ns();
                    while (ld_acquire(c) < need) {
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
        // the neighbours' stores (generic proxy) before this warp's TMA reads (async proxy)
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const int deg = w.pass < g.full ? g.bt : g.rdeg[w.pass - g.full];
        const int np = g.passes;
        const int src = w.pass == 0 ? 0 : (((np - w.pass) % 2 == 0) ? 1 : 2);
        float *dst = g.buf[((np - 1 - w.pass) % 2 == 0) ? 1 : 2];
        Tile2D tg;
        tg.src = g.buf[src];
        tg.total = g.pitch * (g.ny + 2 * g.radius);
        tg.pitch = g.pitch;
        tg.ny = g.ny;
        tg.nx = g.nx;
        tg.x0 = g.radius - g.lead + w.xt * g.stride;
        tg.sc0 = max(g.radius, tg.x0 + g.lead);
        tg.sc1 = min(g.nx + g.radius, tg.x0 + g.lead + g.stride);
        tg.y0 = g.radius + w.sb * g.hsn;
        tg.y1 = min(tg.y0 + g.hsn, g.ny + g.radius);
        tg.stall = 0;
        const CUtensorMap *map = &g.map[src];
        bool done;
        switch (g.cls) {
        case 0: done = batch_dispatch_deg<SH_STAR, 1>(deg, g.v, tg, map, dst, status, ring, g.coeffs); break;
        case 1: done = batch_dispatch_deg<SH_STAR, 2>(deg, g.v, tg, map, dst, status, ring, g.coeffs); break;
        case 2: done = batch_dispatch_deg<SH_BOX, 1>(deg, g.v, tg, map, dst, status, ring, g.coeffs); break;
        default: done = batch_dispatch_deg<SH_BOX, 2>(deg, g.v, tg, map, dst, status, ring, g.coeffs); break;
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

// dst halos := in halos for every grid (out, and scratch when it is used).
__global__ void batch_halo_kernel(const BatchGrid *__restrict__ grids)
{
    const BatchGrid &g = grids[blockIdx.y];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 8 + warp;
    const int R = g.radius, nyp = g.ny + 2 * R, nxp = g.pitch;
    if (row >= nyp || g.passes == 0) return;
    const float *src = g.buf[0] + (size_t)row * nxp;
    const bool full = row < R || row >= nyp - R;
    for (int b = 1; b <= (g.passes > 1 ? 2 : 1); ++b) {
        float *d = g.buf[b] + (size_t)row * nxp;
        if (full) {
            for (int x = lane; x < nxp; x += 32) d[x] = src[x];
        } else if (lane < 2 * R) {
            const int x = lane < R ? lane : nxp - 2 * R + lane;
            d[x] = src[x];
        }
    }
}

}  // namespace an5d

using namespace an5d;

// ---------------------------------------------------------------------------
// Host side.

struct an5d_batch_plan {
    int n;
    std::vector<BatchGrid> grids;        // host copy (maps filled at run time)
    std::vector<an5d_grid_desc> descs;
    std::vector<std::vector<double>> coeffs;
    std::vector<BatchItem> items;
    int class_bt[BATCH_CLASSES] = {8, 4, 4, 2};
    int class_v[BATCH_CLASSES] = {4, 4, 4, 4};  // cells per lane of each class's tiles
    int device = 0, sms = 0;
    void *scratch = nullptr;             // all grids' scratch buffers
    std::vector<size_t> scratch_off;
    BatchGrid *d_grids = nullptr;
    BatchGrid *h_grids = nullptr;        // pinned staging for the table
    BatchItem *d_items = nullptr;
    int *d_counters = nullptr;           // tile counters, then queue, abort, status
    int n_counters = 0;
    int ctas = 0;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    std::vector<const void *> last_in;
    std::vector<void *> last_out;
    double cell_updates = 0;
    int stall_test = 0;                  // fault injection (tests only)
    std::string err;
};

static thread_local std::string g_batch_err;

static int bfail(int st, const std::string &m)
{
    g_batch_err = m;
    return st;
}

static PFN_cuTensorMapEncodeTiled_v12000 batch_encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

static int batch_cls(an5d_shape shape, int radius) { return (shape == AN5D_STAR ? 0 : 2) + (radius - 1); }

// Geometry, passes, items and counters for the current per-class degrees.
static void batch_layout(an5d_batch_plan *bp)
{
    bp->items.clear();
    int counter = 0;
    int max_passes = 0;
    bp->cell_updates = 0;
    for (int i = 0; i < bp->n; ++i) {
        const an5d_grid_desc &d = bp->descs[i];
        BatchGrid &g = bp->grids[i];
        const int R = d.radius;
        g.radius = R;
        g.cls = batch_cls(d.shape, R);
        g.ny = (int)d.ny;
        g.nx = (int)d.nx;
        g.pitch = (int)d.nx + 2 * R;
        int bt = bp->class_bt[g.cls];
        g.bt = bt;
        g.full = (int)(d.T / bt);
        // the remaining T mod bT steps, greedily in the largest built degrees
        int left = (int)(d.T % bt);
        g.rem = 0;
        for (int i = BATCH_MENU - 1; i >= 0; --i)
            while (batch_menu(g.cls, i) < bt && left >= batch_menu(g.cls, i)) {
                g.rdeg[g.rem++] = batch_menu(g.cls, i);
                left -= batch_menu(g.cls, i);
            }
        g.passes = g.full + g.rem;
        g.lead = bt * R;
        g.v = (bp->class_v[g.cls] == BATCH_WIDE_V && bt == batch_wide_deg(g.cls)) ? BATCH_WIDE_V : CELLS_PER_LANE;
        g.stride = 32 * g.v - 2 * bt * R;
        g.tiles_x = (g.nx + g.stride - 1) / g.stride;
        // stream blocks of at most 256 rows (and at least bT*R rows)
        g.nsb = std::max(1, (g.ny + 255) / 256);
        g.hsn = (g.ny + g.nsb - 1) / g.nsb;
        g.hsn = std::max(g.hsn, std::min(g.ny, bt * R));
        g.nsb = (g.ny + g.hsn - 1) / g.hsn;
        g.counter_base = counter;
        counter += g.tiles_x * g.nsb;
        max_passes = std::max(max_passes, g.passes);
        bp->cell_updates += (double)d.ny * d.nx * d.T;
    }
    // Pass-major; inside a pass, grouped by (class, degree) so that the warps
    // running at the same time share the same code (each class and degree is
    // a separate, fully unrolled instantiation).  An item's dependencies (the
    // same grid, pass p - 1) come earlier in the queue.
    auto degree_at = [](const BatchGrid &g, int p) { return p < g.full ? g.bt : g.rdeg[p - g.full]; };
    for (int p = 0; p < max_passes; ++p)
        for (int cls = 0; cls < BATCH_CLASSES; ++cls)
            for (int m = BATCH_MENU - 1; m >= 0; --m)
                for (int i = 0; i < bp->n; ++i) {
                    const BatchGrid &g = bp->grids[i];
                    if (p >= g.passes || g.cls != cls || degree_at(g, p) != batch_menu(cls, m)) continue;
                    for (int sb = 0; sb < g.nsb; ++sb)
                        for (int xt = 0; xt < g.tiles_x; ++xt) bp->items.push_back(BatchItem{i, xt, sb, p});
                }
    bp->n_counters = counter;
}

static int batch_upload_layout(an5d_batch_plan *bp)
{
    cudaFree(bp->d_items);
    cudaFree(bp->d_counters);
    bp->d_items = nullptr;
    bp->d_counters = nullptr;
    if (!bp->items.empty() &&
        cudaMalloc(&bp->d_items, sizeof(BatchItem) * bp->items.size()) != cudaSuccess)
        return bfail(AN5D_ERR_OOM, "batch items");
    if (cudaMalloc(&bp->d_counters, sizeof(int) * (bp->n_counters + 3)) != cudaSuccess)
        return bfail(AN5D_ERR_OOM, "batch counters");
    if (!bp->items.empty() &&
        cudaMemcpy(bp->d_items, bp->items.data(), sizeof(BatchItem) * bp->items.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(AN5D_ERR_CUDA, "batch items upload");
    cudaMemset(bp->d_counters, 0, sizeof(int) * (bp->n_counters + 3));
    if (bp->graph) {
        cudaGraphExecDestroy(bp->graph);
        bp->graph = nullptr;
    }
    bp->last_in.clear();
    bp->last_out.clear();
    return AN5D_OK;
}

extern "C" const char *an5d_batch_last_error(void) { return g_batch_err.c_str(); }

extern "C" an5d_batch_plan *an5d_batch_plan_create(int n, const an5d_grid_desc *descs)
{
    if (n < 1 || !descs) {
        bfail(AN5D_ERR_INVALID_ARG, "n must be >= 1 and descs non-NULL");
        return nullptr;
    }
    for (int i = 0; i < n; ++i) {
        const an5d_grid_desc &d = descs[i];
        if ((d.shape != AN5D_STAR && d.shape != AN5D_BOX) || d.radius < 1 || d.radius > 2 || !d.coeffs ||
            d.ny < 1 || d.nx < 1 || d.T < 0 || (d.ny + 2 * d.radius) * (d.nx + 2 * d.radius) >= (1ll << 31)) {
            bfail(AN5D_ERR_INVALID_ARG, "grid " + std::to_string(i) +
                                            ": shape star/box, radius 1-2, extents >= 1, T >= 0, "
                                            "fewer than 2^31 padded cells");
            return nullptr;
        }
    }
    an5d_batch_plan *bp = new an5d_batch_plan();
    bp->n = n;
    bp->descs.assign(descs, descs + n);
    bp->grids.resize(n);
    bp->coeffs.resize(n);
    for (int i = 0; i < n; ++i) {
        const int nc = an5d_coeff_count(2, descs[i].shape, descs[i].radius);
        bp->coeffs[i].assign(descs[i].coeffs, descs[i].coeffs + nc);
        bp->descs[i].coeffs = bp->coeffs[i].data();
        memset(&bp->grids[i], 0, sizeof(BatchGrid));
        for (int k = 0; k < nc; ++k) bp->grids[i].coeffs[k] = (float)descs[i].coeffs[k];
    }
    size_t off = 0;
    bp->scratch_off.resize(n);
    for (int i = 0; i < n; ++i) {
        bp->scratch_off[i] = off;
        off += ((size_t)(descs[i].ny + 2 * descs[i].radius) * (descs[i].nx + 2 * descs[i].radius) * 4 + 255) / 256 * 256;
    }
    cudaError_t e = cudaGetDevice(&bp->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&bp->sms, cudaDevAttrMultiProcessorCount, bp->device);
    if (e == cudaSuccess) e = cudaMalloc(&bp->scratch, std::max<size_t>(off, 256));
    if (e == cudaSuccess) e = cudaMalloc(&bp->d_grids, sizeof(BatchGrid) * n);
    if (e == cudaSuccess) e = cudaMallocHost(&bp->h_grids, sizeof(BatchGrid) * n);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BATCH_SMEM);
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, BATCH_WARPS * 32, BATCH_SMEM);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bp->graph_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        bfail(e == cudaErrorMemoryAllocation ? AN5D_ERR_OOM : AN5D_ERR_CUDA,
              std::string("batch plan setup: ") + cudaGetErrorString(e));
        an5d_batch_plan_destroy(bp);
        return nullptr;
    }
    bp->ctas = std::max(1, per_sm) * bp->sms;   // persistent: exactly the resident CTAs
    batch_layout(bp);
    if (batch_upload_layout(bp)) {
        an5d_batch_plan_destroy(bp);
        return nullptr;
    }
    return bp;
}

extern "C" void an5d_batch_plan_destroy(an5d_batch_plan *bp)
{
    if (!bp) return;
    cudaDeviceSynchronize();
    if (bp->graph) cudaGraphExecDestroy(bp->graph);
    if (bp->graph_stream) cudaStreamDestroy(bp->graph_stream);
    cudaFree(bp->scratch);
    cudaFree(bp->d_grids);
    cudaFreeHost(bp->h_grids);
    cudaFree(bp->d_items);
    cudaFree(bp->d_counters);
    delete bp;
}

extern "C" int an5d_batch_set_degrees(an5d_batch_plan *bp, const int *class_bt)
{
    if (!bp || !class_bt) return bfail(AN5D_ERR_INVALID_ARG, "NULL argument");
    for (int c = 0; c < BATCH_CLASSES; ++c) {
        bool built = false;
        for (int i = 0; i < BATCH_MENU; ++i) built |= class_bt[c] == batch_menu(c, i);
        if (!built) return bfail(AN5D_ERR_UNSUPPORTED, "degree " + std::to_string(class_bt[c]) +
                                                           " not built for class " + std::to_string(c));
    }
    cudaDeviceSynchronize();
    for (int c = 0; c < BATCH_CLASSES; ++c) bp->class_bt[c] = class_bt[c];
    batch_layout(bp);
    return batch_upload_layout(bp);
}

extern "C" int an5d_batch_set_tiles(an5d_batch_plan *bp, const int *class_tile_x)
{
    if (!bp || !class_tile_x) return bfail(AN5D_ERR_INVALID_ARG, "NULL argument");
    for (int c = 0; c < BATCH_CLASSES; ++c)
        if (class_tile_x[c] != 32 * CELLS_PER_LANE && class_tile_x[c] != 32 * BATCH_WIDE_V)
            return bfail(AN5D_ERR_UNSUPPORTED, "tile width " + std::to_string(class_tile_x[c]) +
                                                   " not built (128 or 192 cells)");
    cudaDeviceSynchronize();
    for (int c = 0; c < BATCH_CLASSES; ++c) bp->class_v[c] = class_tile_x[c] / 32;
    batch_layout(bp);
    return batch_upload_layout(bp);
}

extern "C" int an5d_batch_info(const an5d_batch_plan *bp, an5d_batch_info_t *info)
{
    if (!bp || !info) return AN5D_ERR_INVALID_ARG;
    info->grids = bp->n;
    info->items = (int64_t)bp->items.size();
    info->cell_updates = bp->cell_updates;
    for (int c = 0; c < BATCH_CLASSES; ++c) {
        info->class_bt[c] = bp->class_bt[c];
        // the wide tile applies with the class's wide degree only
        const bool wide = bp->class_v[c] == BATCH_WIDE_V && bp->class_bt[c] == batch_wide_deg(c);
        info->class_tile_x[c] = 32 * (wide ? BATCH_WIDE_V : CELLS_PER_LANE);
    }
    info->ctas = bp->ctas;
    return AN5D_OK;
}

// Per-class degree from the built menu, timed on a 1024^2 grid of the
// class with the single-grid plan (same warp-tile code).
// Time one run of the whole batch (after one untimed run of the same layout).
static int batch_time(an5d_batch_plan *bp, const void *const *ins, void *const *outs, cudaStream_t st,
                      float *ms)
{
    if (int s = an5d_batch_run(bp, ins, outs, st)) return s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    int s = an5d_batch_run(bp, ins, outs, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == AN5D_OK) s = an5d_batch_status(bp);
    return s;
}

extern "C" int an5d_batch_tune_run(an5d_batch_plan *bp, const void *const *ins, void *const *outs,
                                   void *stream)
{
    if (!bp || !ins || !outs) return bfail(AN5D_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    bool present[BATCH_CLASSES] = {false, false, false, false};
    for (int i = 0; i < bp->n; ++i) present[batch_cls(bp->descs[i].shape, bp->descs[i].radius)] = true;
    int best[BATCH_CLASSES], best_v[BATCH_CLASSES];
    for (int c = 0; c < BATCH_CLASSES; ++c) {
        best[c] = bp->class_bt[c];
        best_v[c] = bp->class_v[c];
    }
    auto apply = [&](const int *bt, const int *v) -> int {
        int tx[BATCH_CLASSES];
        for (int c = 0; c < BATCH_CLASSES; ++c) tx[c] = 32 * v[c];
        cudaDeviceSynchronize();
        for (int c = 0; c < BATCH_CLASSES; ++c) bp->class_v[c] = tx[c] / 32;
        return an5d_batch_set_degrees(bp, bt);
    };
    if (int s = apply(best, best_v)) return s;
    float t_best = 0;
    if (int s = batch_time(bp, ins, outs, st, &t_best)) return s;
    // coordinate descent over the classes' (degree, tile width) options,
    // timing the whole batch (the choices interact through the shared queue,
    // so a class is not tuned on a grid of its own)
    for (int sweep = 0; sweep < 2; ++sweep) {
        bool changed = false;
        for (int c = 0; c < BATCH_CLASSES; ++c) {
            if (!present[c]) continue;
            for (int m = 0; m <= BATCH_MENU; ++m) {
                int trial[BATCH_CLASSES], trial_v[BATCH_CLASSES];
                for (int k = 0; k < BATCH_CLASSES; ++k) trial[k] = best[k], trial_v[k] = best_v[k];
                if (m < BATCH_MENU) {
                    trial[c] = batch_menu(c, m);
                    trial_v[c] = CELLS_PER_LANE;
                } else {
                    trial[c] = batch_wide_deg(c);
                    trial_v[c] = BATCH_WIDE_V;
                }
                if (trial[c] == best[c] && trial_v[c] == best_v[c]) continue;
                if (int s = apply(trial, trial_v)) return s;
                float t = 0;
                if (int s = batch_time(bp, ins, outs, st, &t)) return s;
                if (t < t_best) {
                    t_best = t;
                    best[c] = trial[c];
                    best_v[c] = trial_v[c];
                    changed = true;
                }
            }
        }
        if (!changed) break;
    }
    return apply(best, best_v);
}

extern "C" int an5d_batch_tune(an5d_batch_plan *bp, void *stream)
{
    if (!bp) return bfail(AN5D_ERR_INVALID_ARG, "NULL plan");
    // temporary zero-filled inputs and outputs of every grid's padded size
    std::vector<void *> bufs(2 * (size_t)bp->n, nullptr);
    int s = AN5D_OK;
    for (int i = 0; i < bp->n && s == AN5D_OK; ++i) {
        const size_t bytes = (size_t)bp->grids[i].pitch * (bp->grids[i].ny + 2 * bp->grids[i].radius) * 4;
        for (int k = 0; k < 2 && s == AN5D_OK; ++k) {
            if (cudaMalloc(&bufs[2 * i + k], bytes) != cudaSuccess)
                s = bfail(AN5D_ERR_OOM, "batch tune: buffers");
            else
                cudaMemsetAsync(bufs[2 * i + k], 0, bytes, (cudaStream_t)stream);
        }
    }
    if (s == AN5D_OK) {
        std::vector<const void *> ins(bp->n);
        std::vector<void *> outs(bp->n);
        for (int i = 0; i < bp->n; ++i) ins[i] = bufs[2 * i], outs[i] = bufs[2 * i + 1];
        s = an5d_batch_tune_run(bp, ins.data(), outs.data(), stream);
    }
    cudaDeviceSynchronize();
    for (void *b : bufs) cudaFree(b);
    // the captured graph refers to the freed buffers: force a new capture
    if (bp->graph) {
        cudaGraphExecDestroy(bp->graph);
        bp->graph = nullptr;
    }
    bp->last_in.clear();
    bp->last_out.clear();
    return s;
}

extern "C" int an5d_batch_run(an5d_batch_plan *bp, const void *const *ins, void *const *outs, void *stream)
{
    if (!bp || !ins || !outs) return bfail(AN5D_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    auto fn = batch_encode_fn();
    if (!fn) return bfail(AN5D_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    bool same = bp->last_in.size() == (size_t)bp->n;
    for (int i = 0; i < bp->n && same; ++i) same = bp->last_in[i] == ins[i] && bp->last_out[i] == outs[i];
    if (!same) {
        for (int i = 0; i < bp->n; ++i) {
            if (!ins[i] || !outs[i] || (((uintptr_t)ins[i] | (uintptr_t)outs[i]) & 15))
                return bfail(AN5D_ERR_INVALID_ARG, "grid " + std::to_string(i) + ": NULL or misaligned buffer");
            const size_t bytes = (size_t)bp->grids[i].pitch * (bp->grids[i].ny + 2 * bp->grids[i].radius) * 4;
            const char *x = (const char *)ins[i], *y = (const char *)outs[i];
            if (x < y + bytes && y < x + bytes)
                return bfail(AN5D_ERR_ALIAS, "grid " + std::to_string(i) + ": out overlaps in");
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) return bfail(AN5D_ERR_CUDA, "sync");
        for (int i = 0; i < bp->n; ++i) {
            BatchGrid &g = bp->grids[i];
            g.buf[0] = (float *)ins[i];
            g.buf[1] = (float *)outs[i];
            g.buf[2] = (float *)((char *)bp->scratch + bp->scratch_off[i]);
            const cuuint64_t total = (cuuint64_t)g.pitch * (g.ny + 2 * g.radius);
            for (int b = 0; b < 3; ++b) {
                cuuint64_t dim[1] = {total}, strides[1] = {0};
                cuuint32_t box[1] = {32 * CELLS_PER_LANE + 4}, es[1] = {1};
                CUresult r = fn(&g.map[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 1, g.buf[b], dim, strides, box, es,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) return bfail(AN5D_ERR_CUDA, "tensor map encode failed");
            }
            bp->h_grids[i] = g;
        }
        if (cudaMemcpyAsync(bp->d_grids, bp->h_grids, sizeof(BatchGrid) * bp->n, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
            return bfail(AN5D_ERR_CUDA, "grid table upload");
        bp->last_in.assign(ins, ins + bp->n);
        bp->last_out.assign(outs, outs + bp->n);
    }
    for (int i = 0; i < bp->n; ++i)
        if (bp->grids[i].passes == 0) {
            const size_t bytes = (size_t)bp->grids[i].pitch * (bp->grids[i].ny + 2 * bp->grids[i].radius) * 4;
            if (cudaMemcpyAsync(outs[i], ins[i], bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return bfail(AN5D_ERR_CUDA, "T = 0 copy");
        }
    if (!bp->graph) {
        // capture: reset queue/counters, halo copies, the persistent sweep
        cudaStream_t cs = bp->graph_stream;
        cudaGraph_t g = nullptr;
        int maxrows = 0;
        for (const auto &x : bp->grids) maxrows = std::max(maxrows, x.ny + 2 * x.radius);
        int *queue = bp->d_counters + bp->n_counters;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return bfail(AN5D_ERR_CUDA, "graph capture begin");
        cudaMemsetAsync(bp->d_counters, 0, sizeof(int) * (bp->n_counters + 3), cs);
        batch_halo_kernel<<<dim3((maxrows + 7) / 8, bp->n), 256, 0, cs>>>(bp->d_grids);
        batch_kernel<<<bp->ctas, BATCH_WARPS * 32, BATCH_SMEM, cs>>>(bp->d_grids, bp->d_items, (int)bp->items.size(),
                                                                   queue, bp->d_counters, queue + 2, queue + 1,
                                                                   bp->stall_test ? (int)bp->items.size() - 1 : -1);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&bp->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(AN5D_ERR_CUDA, std::string("graph: ") + cudaGetErrorString(e));
    }
    if (cudaGraphLaunch(bp->graph, st) != cudaSuccess) return bfail(AN5D_ERR_CUDA, "graph launch");
    return AN5D_OK;
}

extern "C" int an5d_batch_status(an5d_batch_plan *bp)
{
    if (!bp) return AN5D_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return bfail(AN5D_ERR_CUDA, "sync");
    int h[3] = {0, 0, 0};
    cudaMemcpy(h, bp->d_counters + bp->n_counters, sizeof(h), cudaMemcpyDeviceToHost);
    if (h[2] & STATUS_TIMEOUT) return bfail(AN5D_ERR_TIMEOUT, "a bounded device wait gave up");
    if (h[1]) return bfail(AN5D_ERR_TIMEOUT, "the batch was aborted");
    return AN5D_OK;
}

extern "C" int an5d_batch_inject_stall(an5d_batch_plan *bp, int enable)
{
    if (!bp) return bfail(AN5D_ERR_INVALID_ARG, "NULL plan");
    bp->stall_test = enable ? 1 : 0;
    if (bp->graph) {               // the flag is a kernel argument: re-capture
        cudaGraphExecDestroy(bp->graph);
        bp->graph = nullptr;
    }
    return AN5D_OK;
}
