// an5d_api.cu -- the C ABI declared in include/an5d.h: plans, the pass loop
// of the host code (AN5D Section 3.3), the analytic model and the autotuner.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "an5d.h"
#include "an5d_internal.h"
#include "model.h"

namespace an5d {

std::vector<KernelEntry> &registry()
{
    static std::vector<KernelEntry> r;
    return r;
}

const KernelEntry *find_kernel(const KernelKey &k)
{
    for (const auto &e : registry())
        if (e.key == k) return &e;
    return nullptr;
}

// ---------------------------------------------------------------------------
// Thread-local error reporting.

static thread_local std::string g_err = "";
static thread_local int g_status = AN5D_OK;

static int fail(int status, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    g_status = status;
    return status;
}

static int ok()
{
    g_status = AN5D_OK;
    return AN5D_OK;
}

#define CUDA_TRY(expr)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? AN5D_ERR_OOM : AN5D_ERR_CUDA,     \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// ---------------------------------------------------------------------------
// Tensor-map encoding through the driver entry point (no -lcuda needed).

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

static size_t elem_size(int dtype)
{
    switch (dtype) {
    case DT_F64: return 8;
    case DT_F16S: return 2;
    default: return 4;
    }
}

// 1D tiled map over a whole padded array; box = tile + alignment slack.
static int encode_row_map(CUtensorMap *m, const void *base, int dtype, int64_t total, int box)
{
    auto fn = encode_fn();
    if (!fn) return fail(AN5D_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
    CUtensorMapDataType t = dtype == DT_F64    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                            : dtype == DT_F16S ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t dim[1] = {(cuuint64_t)total};
    cuuint32_t boxd[1] = {(cuuint32_t)box};
    cuuint32_t es[1] = {1};
    cuuint64_t no_strides[1] = {0};  // rank 1 has no strides, but the driver wants a pointer
    CUresult r = fn(m, t, 1, const_cast<void *>(base), dim, no_strides, boxd, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(AN5D_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return AN5D_OK;
}

// ---------------------------------------------------------------------------
// Halo copy: dst's halo := src's halo (one CTA per padded x row).

template <typename W>
__global__ void halo_copy_kernel(const W *__restrict__ src, W *__restrict__ dst, int nzp, int nyp,
                                 int nxp, int hz, int R)
{
    const int row = blockIdx.x;
    const int z = row / nyp, y = row % nyp;
    const bool full = z < hz || z >= nzp - hz || y < R || y >= nyp - R;
    const size_t base = (size_t)row * nxp;
    if (full) {
        for (int x = threadIdx.x; x < nxp; x += blockDim.x) dst[base + x] = src[base + x];
    } else {
        for (int x = threadIdx.x; x < 2 * R; x += blockDim.x) {
            const int xx = x < R ? x : nxp - 2 * R + x;
            dst[base + xx] = src[base + xx];
        }
    }
}

}  // namespace an5d

using namespace an5d;

// ---------------------------------------------------------------------------
// Plan.

struct an5d_plan {
    int ndim, shape, radius, dtype;
    int64_t dims[3];      // interior extents, slowest first (ndim entries used)
    int64_t nz, ny, nx;   // interior extents as 3D (nz = 1 in 2D)
    int64_t total;        // padded elements
    size_t bytes;         // padded bytes
    int n;                // coefficients
    double coeffs[MAX_COEFFS];  // rounded to the compute precision
    int post = POST_NONE; // per-step division (division-type stencils)
    double post_c = 0;    // divisor or reciprocal, rounded to the compute precision
    int device;
    int sms;
    void *scratch = nullptr;
    int *d_status = nullptr;
    void *stage_in = nullptr, *stage_out = nullptr;
    int bt = 1;
    int hsn = 0;
    int tile = 0;         // tile variant of the sweep kernel (0 = default width)
    // 3D: second stream and fork/join events on which a pass's narrow last
    // column runs beside the main launch (null: the two run one after the other)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double model_gcells = 0, measured_gcells = 0;
    int bt_max = 0;
    int stall_test = 0;  // fault injection (tests only)
    void *work = nullptr;  // reusable work memory of the adjoint (grown on demand)
    size_t work_bytes = 0;
};

extern "C" const char *an5d_version(void) { return "an5d-gb300 0.1 (sm_103a)"; }
extern "C" const char *an5d_last_error(void) { return g_err.c_str(); }
extern "C" int an5d_last_status(void) { return g_status; }

extern "C" int an5d_coeff_count(int ndim, an5d_shape shape, int radius)
{
    if (ndim != 2 && ndim != 3) return fail(AN5D_ERR_UNSUPPORTED, "ndim must be 2 or 3");
    if (radius < 1 || radius > 4) return fail(AN5D_ERR_UNSUPPORTED, "radius must be in 1..4");
    if (shape == AN5D_STAR) return 2 * ndim * radius + 1;
    if (shape == AN5D_BOX) {
        int n = 1;
        for (int i = 0; i < ndim; ++i) n *= 2 * radius + 1;
        return n;
    }
    return fail(AN5D_ERR_INVALID_ARG, "shape must be AN5D_STAR or AN5D_BOX");
}

static int largest_bt(const an5d_plan *p)
{
    int best = 0;
    for (const auto &e : registry())
        if (e.key.ndim == p->ndim && e.key.shape == p->shape && e.key.radius == p->radius &&
            e.key.dtype == p->dtype && e.key.post == p->post)
            best = std::max(best, e.key.bt);
    return best;
}

// Geometry of one pass with degree bt.
struct PassGeom {
    const KernelEntry *k;
    int tile_stride_x, tiles_x, tile_stride_y, tiles_y, hsn, stream_blocks, units, ctas;
    // padded column where tile column 0's compute region starts, chosen so
    // that tiles start on even columns (the sweeps move 8-byte pairs when
    // rows and tiles are even): R rounded down to even in 2D, R or R - 1 in
    // 3D; a halo column the first tile takes in is never stored
    int x_base;
    // 3D: a narrow kernel for the last tile column when the main tiles leave a
    // ragged remainder that fits it (tail_k null otherwise): main columns
    // cover [x_base, x_base + tiles_x * tile_stride_x), the narrow one the rest
    const KernelEntry *tail_k;
    int tail_stride_x, tail_units;
};

// Kernel of degree bt in tile variant `tile`, or (tile < 0) in the plan's
// variant, where a degree the variant does not build (a remainder pass)
// runs on the default kernel.
static const KernelEntry *plan_kernel(const an5d_plan *p, int bt, int tile)
{
    if (tile >= 0) return find_kernel(KernelKey{p->ndim, p->shape, p->radius, p->dtype, bt, p->post, tile});
    const KernelEntry *k = find_kernel(KernelKey{p->ndim, p->shape, p->radius, p->dtype, bt, p->post, p->tile});
    if (!k && p->tile) k = find_kernel(KernelKey{p->ndim, p->shape, p->radius, p->dtype, bt, p->post, 0});
    return k;
}

// Tile variants built for the plan's stencil (0, the default, first).
static std::vector<int> tile_variants(const an5d_plan *p)
{
    std::vector<int> t{0};
    for (const auto &e : registry())
        if (e.key.ndim == p->ndim && e.key.shape == p->shape && e.key.radius == p->radius &&
            e.key.dtype == p->dtype && e.key.post == p->post &&
            std::find(t.begin(), t.end(), e.key.tile) == t.end())
            t.push_back(e.key.tile);
    std::sort(t.begin() + 1, t.end());
    return t;
}

static bool variant_has(const an5d_plan *p, int tile, int bt)
{
    return find_kernel(KernelKey{p->ndim, p->shape, p->radius, p->dtype, bt, p->post, tile}) != nullptr;
}

static int pass_geometry(const an5d_plan *p, int bt, int hsn_req, PassGeom *g, int tile = -1)
{
    g->k = plan_kernel(p, bt, tile);
    if (!g->k)
        return fail(AN5D_ERR_UNSUPPORTED, "no kernel for ndim=%d shape=%d R=%d dtype=%d bT=%d",
                    p->ndim, p->shape, p->radius, p->dtype, bt);
    const int R = p->radius;
    g->tile_stride_x = g->k->tile_x - 2 * bt * R;
    // Tiles start on even columns (the tile origin is x_base - bT R; tile
    // widths and strides are even), so that with an even pitch every row a
    // lane reads or writes starts on an 8-byte boundary.  The first compute
    // region may then start one column early, on a halo column it never stores.
    g->x_base = p->ndim == 2 ? (R & ~1) : R - ((R * (bt - 1)) & 1);
    g->tiles_x = (int)((p->nx + R - g->x_base + g->tile_stride_x - 1) / g->tile_stride_x);
    g->tail_k = nullptr;
    g->tail_stride_x = 0;
    g->tail_units = 0;
    if (p->ndim == 3) {
        g->tile_stride_y = g->k->tile_y - 2 * bt * R;
        g->tiles_y = (int)((p->ny + g->tile_stride_y - 1) / g->tile_stride_y);
        // a ragged last column that one narrow tile covers runs on the
        // narrow kernel (same tile rows) instead of a mostly idle full tile
        KernelKey tk{p->ndim, p->shape, p->radius, p->dtype, bt, p->post, 0};
        tk.part = 1;
        const KernelEntry *t = find_kernel(tk);
        const int64_t span = p->nx + R - g->x_base;  // columns the tiles cover
        const int64_t full = span / g->tile_stride_x, rest = span - full * g->tile_stride_x;
        if (t && t->tile_y == g->k->tile_y && full >= 1 && rest > 0 &&
            rest <= t->tile_x - 2 * bt * R) {
            g->tail_k = t;
            g->tail_stride_x = t->tile_x - 2 * bt * R;
            g->tiles_x = (int)full;
        }
    } else {
        g->tile_stride_y = 1;
        g->tiles_y = 1;
    }
    const int64_t slen = p->ndim == 3 ? p->nz : p->ny;
    int hsn = hsn_req > 0 ? hsn_req : (int)slen;
    hsn = (int)std::min<int64_t>(std::max(1, hsn), slen);
    g->hsn = hsn;
    g->stream_blocks = (int)((slen + hsn - 1) / hsn);
    const int64_t units = (int64_t)g->tiles_x * g->tiles_y * g->stream_blocks;
    if (units > (1ll << 30)) return fail(AN5D_ERR_UNSUPPORTED, "grid too large");
    g->units = (int)units;
    g->ctas = (g->units + g->k->units_per_cta - 1) / g->k->units_per_cta;
    if (g->tail_k) g->tail_units = g->tiles_y * g->stream_blocks;  // one CTA per tail tile
    return AN5D_OK;
}

// Resident work units per SM for a kernel (occupancy query).
static int resident_units(const KernelEntry *k)
{
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k->func, k->threads,
                                                      k->smem_bytes) != cudaSuccess)
        blocks = 1;
    if (k->smem_bytes > 48 * 1024) {
        // the attribute may not be set yet: estimate from shared memory alone
        cudaFuncSetAttribute(k->func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)k->smem_bytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k->func, k->threads, k->smem_bytes);
    }
    return std::max(1, blocks) * k->units_per_cta;
}

// Stream-block length that makes the pass one (or `waves`) full wave(s).
static int default_hsn(const an5d_plan *p, int bt, int waves)
{
    PassGeom g;
    if (pass_geometry(p, bt, 0, &g)) return 0;
    const int64_t cap = (int64_t)resident_units(g.k) * p->sms * waves;
    const int64_t tiles = (int64_t)g.tiles_x * g.tiles_y;
    const int64_t slen = p->ndim == 3 ? p->nz : p->ny;
    int64_t nsb = std::max<int64_t>(1, cap / std::max<int64_t>(1, tiles));
    nsb = std::min(nsb, slen);
    return (int)((slen + nsb - 1) / nsb);
}

static double model_for(const an5d_plan *p, int bt, int hsn)
{
    PassGeom g;
    if (pass_geometry(p, bt, hsn, &g)) return 0.0;
    ModelInput mi;
    mi.ndim = p->ndim;
    mi.shape = p->shape;
    mi.radius = p->radius;
    mi.dtype = p->dtype;
    mi.bt = bt;
    mi.nz = p->nz;
    mi.ny = p->ny;
    mi.nx = p->nx;
    mi.tile_x = g.k->tile_x;
    mi.tile_y = g.k->tile_y;
    mi.tiles_x = g.tiles_x;
    mi.tiles_y = g.tiles_y;
    mi.hsn = g.hsn;
    mi.stream_blocks = g.stream_blocks;
    mi.units = g.units;
    mi.resident_units = resident_units(g.k) * p->sms;
    mi.sms = p->sms;
    return model_gcells(mi);
}

static void choose_default(an5d_plan *p)
{
    double best = -1.0;
    int bbt = 1, bh = 0, btile = 0;
    for (int tile : tile_variants(p)) {
        p->tile = tile;
        for (int bt = 1; bt <= p->bt_max; ++bt) {
            if (!variant_has(p, tile, bt)) continue;
            const int h = default_hsn(p, bt, 1);
            const double m = model_for(p, bt, h);
            if (m > best) {
                best = m;
                bbt = bt;
                bh = h;
                btile = tile;
            }
        }
    }
    p->tile = btile;
    p->bt = bbt;
    p->hsn = bh;
    p->model_gcells = best;
    p->measured_gcells = 0.0;
}

static an5d_plan *plan_create_impl(int ndim, an5d_shape shape, int radius, const double *coeffs,
                                   an5d_dtype dtype, const int64_t *dims, int post, double post_c)
{
    int n = an5d_coeff_count(ndim, shape, radius);
    if (n < 0) return nullptr;
    if (n > MAX_COEFFS) {
        fail(AN5D_ERR_UNSUPPORTED, "%d coefficients exceed the library's %d", n, MAX_COEFFS);
        return nullptr;
    }
    if (!coeffs || !dims) {
        fail(AN5D_ERR_INVALID_ARG, "coeffs and dims must not be NULL");
        return nullptr;
    }
    if (dtype < AN5D_F32 || dtype > AN5D_F32_COMPENSATED) {
        fail(AN5D_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
        return nullptr;
    }
    int64_t total = 1;
    for (int i = 0; i < ndim; ++i) {
        if (dims[i] < 1 || dims[i] > (1ll << 30)) {
            fail(AN5D_ERR_INVALID_ARG, "dims[%d] = %lld out of range", i, (long long)dims[i]);
            return nullptr;
        }
        total *= dims[i] + 2 * radius;
        if (total >= (1ll << 31)) {
            fail(AN5D_ERR_UNSUPPORTED, "padded array must have fewer than 2^31 elements");
            return nullptr;
        }
    }
    an5d_plan *p = new an5d_plan();
    p->ndim = ndim;
    p->shape = shape;
    p->radius = radius;
    p->dtype = dtype;
    p->n = n;
    for (int i = 0; i < 3; ++i) p->dims[i] = i < ndim ? dims[i] : 0;
    p->nz = ndim == 3 ? dims[0] : 1;
    p->ny = dims[ndim - 2];
    p->nx = dims[ndim - 1];
    p->total = total;
    p->bytes = (size_t)total * elem_size(dtype);
    const bool dbl = dtype == AN5D_F64;
    for (int k = 0; k < n; ++k) p->coeffs[k] = dbl ? coeffs[k] : (double)(float)coeffs[k];
    p->post = post;
    p->post_c = post_c;
    p->bt_max = largest_bt(p);
    if (p->bt_max == 0) {
        fail(AN5D_ERR_UNSUPPORTED, "stencil ndim=%d shape=%d R=%d dtype=%d post=%d is not built",
             ndim, (int)shape, radius, (int)dtype, post);
        delete p;
        return nullptr;
    }
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&p->scratch, p->bytes);
    if (e == cudaSuccess && ndim == 3) e = cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess && ndim == 3) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && ndim == 3) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        fail(e == cudaErrorMemoryAllocation ? AN5D_ERR_OOM : AN5D_ERR_CUDA, "plan setup: %s",
             cudaGetErrorString(e));
        cudaFree(p->d_status);
        cudaFree(p->scratch);
        if (p->aux) cudaStreamDestroy(p->aux);
        if (p->ev_fork) cudaEventDestroy(p->ev_fork);
        if (p->ev_join) cudaEventDestroy(p->ev_join);
        delete p;
        return nullptr;
    }
    choose_default(p);
    ok();
    return p;
}

extern "C" an5d_plan *an5d_plan_create(int ndim, an5d_shape shape, int radius,
                                       const double *coeffs, an5d_dtype dtype,
                                       const int64_t *dims)
{
    return plan_create_impl(ndim, shape, radius, coeffs, dtype, dims, POST_NONE, 0.0);
}

extern "C" an5d_plan *an5d_plan_create_div(int ndim, an5d_shape shape, int radius,
                                           const double *coeffs, double divisor, an5d_post post,
                                           an5d_dtype dtype, const int64_t *dims)
{
    if (post != AN5D_POST_DIV && post != AN5D_POST_MUL_RCP) {
        fail(AN5D_ERR_INVALID_ARG, "post must be AN5D_POST_DIV or AN5D_POST_MUL_RCP");
        return nullptr;
    }
    if (dtype != AN5D_F32 && dtype != AN5D_F64) {
        fail(AN5D_ERR_UNSUPPORTED, "division-type stencils are built for FP32 and FP64 only");
        return nullptr;
    }
    // the divisor and its reciprocal, each rounded once to the compute precision
    double c;
    if (dtype == AN5D_F32) {
        const float d = (float)divisor;
        c = post == AN5D_POST_DIV ? (double)d : (double)(1.0f / d);
    } else {
        c = post == AN5D_POST_DIV ? divisor : 1.0 / divisor;
    }
    if (!std::isfinite(divisor) || divisor == 0.0 || !std::isfinite(c) || c == 0.0) {
        fail(AN5D_ERR_INVALID_ARG, "divisor must be finite and nonzero, with a nonzero reciprocal");
        return nullptr;
    }
    return plan_create_impl(ndim, shape, radius, coeffs, dtype, dims,
                            post == AN5D_POST_DIV ? POST_DIV : POST_MUL, c);
}

extern "C" void an5d_plan_destroy(an5d_plan *p)
{
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    cudaFree(p->scratch);
    cudaFree(p->d_status);
    cudaFree(p->stage_in);
    cudaFree(p->stage_out);
    cudaFree(p->work);
    if (p->aux) cudaStreamDestroy(p->aux);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (cur >= 0) cudaSetDevice(cur);
    delete p;
}

extern "C" int an5d_plan_config(const an5d_plan *p, an5d_config *cfg)
{
    if (!p || !cfg) return fail(AN5D_ERR_INVALID_ARG, "NULL plan or cfg");
    PassGeom g;
    if (int s = pass_geometry(p, p->bt, p->hsn, &g)) return s;
    cfg->bT = p->bt;
    cfg->tile_x = g.k->tile_x;
    cfg->tile_y = g.k->tile_y;
    cfg->stream_axis = 0;
    cfg->hsn = g.hsn;
    cfg->warps_per_cta = g.k->threads / 32;
    cfg->ctas = g.ctas + g.tail_units;
    cfg->launches_per_pass = g.tail_k ? 2 : 1;
    cfg->model_gcells = p->model_gcells;
    cfg->measured_gcells = p->measured_gcells;
    return ok();
}

extern "C" int an5d_plan_set_config(an5d_plan *p, int bt, int hsn)
{
    if (!p) return fail(AN5D_ERR_INVALID_ARG, "NULL plan");
    if (bt < 0 || hsn < 0) return fail(AN5D_ERR_INVALID_ARG, "bT and hsn must be >= 0");
    const int nbt = bt > 0 ? bt : p->bt;
    if (!variant_has(p, 0, nbt))
        return fail(AN5D_ERR_UNSUPPORTED, "bT=%d is not built for this stencil", nbt);
    if (!variant_has(p, p->tile, nbt)) p->tile = 0;  // the variant lacks this degree
    p->bt = nbt;
    p->hsn = hsn > 0 ? hsn : default_hsn(p, nbt, 1);
    p->model_gcells = model_for(p, p->bt, p->hsn);
    p->measured_gcells = 0.0;
    return ok();
}

extern "C" int64_t an5d_plan_launches(const an5d_plan *p, int64_t T)
{
    if (!p) return fail(AN5D_ERR_INVALID_ARG, "NULL plan");
    if (T < 0) return fail(AN5D_ERR_INVALID_ARG, "T must be >= 0");
    if (T == 0) return 0;  // one device-to-device copy, no kernel
    const int64_t full = T / p->bt;
    const int rem = (int)(T % p->bt);
    const int64_t np = full + (rem ? 1 : 0);
    int64_t n = np > 1 ? 2 : 1;  // halo copies into out (and into the scratch grid)
    PassGeom g;
    if (full) {
        if (int s = pass_geometry(p, p->bt, p->hsn, &g)) return s;
        n += full * (g.tail_k ? 2 : 1);
    }
    if (rem) {
        if (int s = pass_geometry(p, rem, p->hsn, &g)) return s;
        n += g.tail_k ? 2 : 1;
    }
    ok();
    return n;
}

extern "C" int an5d_plan_set_tile(an5d_plan *p, int tile_x)
{
    if (!p) return fail(AN5D_ERR_INVALID_ARG, "NULL plan");
    if (tile_x < 0) return fail(AN5D_ERR_INVALID_ARG, "tile_x must be >= 0");
    if (tile_x && !variant_has(p, tile_x, p->bt))
        return fail(AN5D_ERR_UNSUPPORTED, "no %d-wide tile variant at bT=%d for this stencil", tile_x, p->bt);
    p->tile = tile_x;
    p->model_gcells = model_for(p, p->bt, p->hsn);
    p->measured_gcells = 0.0;
    return ok();
}

extern "C" int an5d_plan_set_coeffs(an5d_plan *p, const double *coeffs)
{
    if (!p || !coeffs) return fail(AN5D_ERR_INVALID_ARG, "NULL plan or coeffs");
    const bool dbl = p->dtype == AN5D_F64;
    for (int k = 0; k < p->n; ++k) p->coeffs[k] = dbl ? coeffs[k] : (double)(float)coeffs[k];
    return ok();
}

static bool overlaps(const void *a, const void *b, size_t n)
{
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + n && y < x + n;
}

static int launch_halo_copy(const an5d_plan *p, const void *src, void *dst, cudaStream_t st)
{
    const int R = p->radius;
    const int hz = p->ndim == 3 ? R : 0;
    const int nzp = (int)(p->nz + 2 * hz), nyp = (int)(p->ny + 2 * R), nxp = (int)(p->nx + 2 * R);
    const int rows = nzp * nyp;
    switch (elem_size(p->dtype)) {
    case 2:
        halo_copy_kernel<uint16_t><<<rows, 128, 0, st>>>((const uint16_t *)src, (uint16_t *)dst, nzp,
                                                         nyp, nxp, hz, R);
        break;
    case 8:
        halo_copy_kernel<uint64_t><<<rows, 128, 0, st>>>((const uint64_t *)src, (uint64_t *)dst, nzp,
                                                         nyp, nxp, hz, R);
        break;
    default:
        halo_copy_kernel<uint32_t><<<rows, 128, 0, st>>>((const uint32_t *)src, (uint32_t *)dst, nzp,
                                                         nyp, nxp, hz, R);
    }
    CUDA_TRY(cudaGetLastError());
    return AN5D_OK;
}

static int launch_pass(const an5d_plan *p, int bt, const void *src, void *dst, cudaStream_t st)
{
    PassGeom g;
    if (int s = pass_geometry(p, bt, p->hsn, &g)) return s;
    PassDesc d;
    memset(&d, 0, sizeof(d));
    const int A = 16 / (int)elem_size(p->dtype);
    if (int s = encode_row_map(&d.tmap, src, p->dtype, p->total, g.k->tile_x + A)) return s;
    d.dst = dst;
    d.status = p->d_status;
    d.pitch = p->nx + 2 * p->radius;
    d.plane = d.pitch * (p->ny + 2 * p->radius);
    d.nz = (int)p->nz;
    d.ny = (int)p->ny;
    d.nx = (int)p->nx;
    d.tile_stride_x = g.tile_stride_x;
    d.x_base = g.x_base;
    d.tile_stride_y = g.tile_stride_y;
    d.tiles_x = g.tiles_x;
    d.tiles_y = g.tiles_y;
    d.hsn = g.hsn;
    d.stream_blocks = g.stream_blocks;
    d.total_units = g.units;
    d.ctas = g.ctas;
    d.stall_test = p->ndim == 2 ? p->stall_test : 0;
    d.post_c = p->post_c;
    for (int k = 0; k < p->n; ++k) d.coeffs[k] = p->coeffs[k];
    if (!g.tail_k) {
        CUDA_TRY(g.k->launch(d, st));
        return AN5D_OK;
    }
    // the last tile column, on the narrow kernel: its own row box, its tiles
    // start where the main columns' compute regions end.  It writes cells
    // the main launch does not touch, so with the plan's second stream it
    // runs beside the main launch (forked after, and joined before, whatever
    // `st` holds around this pass) and its CTAs fill the main launch's last
    // wave instead of waiting for it.
    PassDesc dt = d;
    if (int s = encode_row_map(&dt.tmap, src, p->dtype, p->total, g.tail_k->tile_x + A)) return s;
    dt.tile_stride_x = g.tail_stride_x;
    dt.x_base = g.x_base + g.tiles_x * g.tile_stride_x;
    dt.tiles_x = 1;
    dt.total_units = g.tail_units;
    dt.ctas = g.tail_units;
    if (p->aux) {
        CUDA_TRY(cudaEventRecord(p->ev_fork, st));
        CUDA_TRY(cudaStreamWaitEvent(p->aux, p->ev_fork, 0));
        CUDA_TRY(g.tail_k->launch(dt, p->aux));
        CUDA_TRY(cudaEventRecord(p->ev_join, p->aux));
        CUDA_TRY(g.k->launch(d, st));
        CUDA_TRY(cudaStreamWaitEvent(st, p->ev_join, 0));
    } else {
        CUDA_TRY(g.k->launch(d, st));
        CUDA_TRY(g.tail_k->launch(dt, st));
    }
    return AN5D_OK;
}

static int run_impl(an5d_plan *p, const void *in, void *out, int64_t T, cudaStream_t st)
{
    if (T == 0) {
        CUDA_TRY(cudaMemcpyAsync(out, in, p->bytes, cudaMemcpyDeviceToDevice, st));
        return ok();
    }
    // Pass list (Section 3.3): floor(T/bT) passes of bT, then one of T mod bT.
    std::vector<int> passes((size_t)(T / p->bt), p->bt);
    if (T % p->bt) passes.push_back((int)(T % p->bt));
    const size_t np = passes.size();
    if (int s = launch_halo_copy(p, in, out, st)) return s;
    if (np > 1)
        if (int s = launch_halo_copy(p, in, p->scratch, st)) return s;
    const void *src = in;
    for (size_t k = 0; k < np; ++k) {
        void *dst = ((np - 1 - k) % 2 == 0) ? out : p->scratch;
        if (int s = launch_pass(p, passes[k], src, dst, st)) return s;
        src = dst;
    }
    return ok();
}

static int check_run_args(an5d_plan *p, const void *in, const void *out, int64_t T)
{
    if (!p) return fail(AN5D_ERR_INVALID_ARG, "NULL plan");
    if (!in || !out) return fail(AN5D_ERR_INVALID_ARG, "NULL in/out");
    if (T < 0) return fail(AN5D_ERR_INVALID_ARG, "T must be >= 0");
    if (((uintptr_t)in | (uintptr_t)out) & 15)
        return fail(AN5D_ERR_INVALID_ARG, "in/out must be 16-byte aligned");
    if (overlaps(in, out, p->bytes)) return fail(AN5D_ERR_ALIAS, "out overlaps in");
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device)
        return fail(AN5D_ERR_INVALID_ARG, "current device %d differs from the plan's device %d", dev,
                    p->device);
    return AN5D_OK;
}

extern "C" int an5d_run(an5d_plan *p, const void *in, void *out, int64_t T, void *stream)
{
    if (int s = check_run_args(p, in, out, T)) return s;
    return run_impl(p, in, out, T, (cudaStream_t)stream);
}

extern "C" int an5d_run_host(an5d_plan *p, const void *in_host, void *out_host, int64_t T,
                             void *stream)
{
    if (!p || !in_host || !out_host) return fail(AN5D_ERR_INVALID_ARG, "NULL argument");
    if (T < 0) return fail(AN5D_ERR_INVALID_ARG, "T must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (!p->stage_in) CUDA_TRY(cudaMalloc(&p->stage_in, p->bytes));
    if (!p->stage_out) CUDA_TRY(cudaMalloc(&p->stage_out, p->bytes));
    CUDA_TRY(cudaMemcpyAsync(p->stage_in, in_host, p->bytes, cudaMemcpyHostToDevice, st));
    if (int s = run_impl(p, p->stage_in, p->stage_out, T, st)) return s;
    CUDA_TRY(cudaMemcpyAsync(out_host, p->stage_out, p->bytes, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return ok();
}

extern "C" int an5d_plan_status(an5d_plan *p)
{
    if (!p) return fail(AN5D_ERR_INVALID_ARG, "NULL plan");
    CUDA_TRY(cudaDeviceSynchronize());
    int h = 0;
    CUDA_TRY(cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(p->d_status, 0, sizeof(int)));
    if (h & STATUS_TIMEOUT) return fail(AN5D_ERR_TIMEOUT, "a bounded device wait gave up");
    return ok();
}

// ---------------------------------------------------------------------------
// Autotuner (Section 5.3 "Tuned": model-ranked candidates, top-k timed).

namespace {
struct TuneKey {
    int ndim, shape, radius, dtype, post, device;
    int64_t nz, ny, nx;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(ndim, shape, radius, dtype, post, device, nz, ny, nx) <
               std::tie(o.ndim, o.shape, o.radius, o.dtype, o.post, o.device, o.nz, o.ny, o.nx);
    }
};
struct TuneVal {
    int bt, hsn, tile;
    double model, measured;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;
}  // namespace

extern "C" int an5d_plan_tune(an5d_plan *p, int topk, int64_t T_probe, void *stream)
{
    if (!p) return fail(AN5D_ERR_INVALID_ARG, "NULL plan");
    if (topk < 1) topk = 1;
    if (T_probe < 1) T_probe = 1;
    TuneKey key{p->ndim, p->shape, p->radius, p->dtype, p->post, p->device, p->nz, p->ny, p->nx};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            p->bt = it->second.bt;
            p->hsn = it->second.hsn;
            p->tile = it->second.tile;
            p->model_gcells = it->second.model;
            p->measured_gcells = it->second.measured;
            return ok();
        }
    }
    struct Cand {
        int bt, hsn, tile;
        double model;
    };
    // the model's top k of every tile variant are timed
    const int save_tile = p->tile;
    std::vector<Cand> cands;
    for (int tile : tile_variants(p)) {
        p->tile = tile;
        std::vector<Cand> vc;
        for (int bt = 1; bt <= p->bt_max; ++bt) {
            if (!variant_has(p, tile, bt)) continue;
            for (int waves = 1; waves <= 4; waves *= 2) {
                const int h = default_hsn(p, bt, waves);
                if (h <= 0) continue;
                bool dup = false;
                for (auto &c : vc) dup |= (c.bt == bt && c.hsn == h);
                if (!dup) vc.push_back({bt, h, tile, model_for(p, bt, h)});
            }
        }
        std::sort(vc.begin(), vc.end(), [](const Cand &a, const Cand &b) { return a.model > b.model; });
        if ((int)vc.size() > topk) vc.resize(topk);
        cands.insert(cands.end(), vc.begin(), vc.end());
    }
    p->tile = save_tile;
    cudaStream_t st = (cudaStream_t)stream;
    void *a = nullptr, *b = nullptr;
    CUDA_TRY(cudaMalloc(&a, p->bytes));
    cudaError_t e = cudaMalloc(&b, p->bytes);
    if (e != cudaSuccess) {
        cudaFree(a);
        return fail(AN5D_ERR_OOM, "tune buffers: %s", cudaGetErrorString(e));
    }
    cudaMemsetAsync(a, 0, p->bytes, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int save_bt = p->bt, save_hsn = p->hsn;
    double best = -1.0;
    Cand win = cands.empty() ? Cand{save_bt, save_hsn, save_tile, 0.0} : cands[0];
    int status = AN5D_OK;
    // one warm-up and one timed run of candidate c; false on a run error
    auto time_cand = [&](const Cand &c) -> bool {
        p->bt = c.bt;
        p->hsn = c.hsn;
        p->tile = c.tile;
        const int64_t T = std::max<int64_t>(T_probe, c.bt);
        if ((status = run_impl(p, a, b, T, st))) return false;   // warm-up
        cudaEventRecord(e0, st);
        if ((status = run_impl(p, a, b, T, st))) return false;
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double g = (double)p->nz * p->ny * p->nx * T / (ms * 1e-3) / 1e9;
        if (g > best) {
            best = g;
            win = c;
        }
        return true;
    };
    for (const auto &c : cands)
        if (!time_cand(c)) break;
    // Refine the winner's stream block by measurement: the model's wave
    // arithmetic only proposes a few lengths, and the measured rate moves by
    // several percent between neighbouring ones (lead-in planes against the
    // fill of the last wave).  Time the block counts around the winner's.
    if (status == AN5D_OK && !cands.empty()) {
        const Cand w0 = win;
        const int64_t slen = p->ndim == 3 ? p->nz : p->ny;
        const int64_t nsb = (slen + w0.hsn - 1) / w0.hsn;
        std::vector<int> tried{w0.hsn};
        for (const auto &c : cands)
            if (c.bt == w0.bt && c.tile == w0.tile) tried.push_back(c.hsn);
        for (double f : {0.5, 0.75, 1.25, 1.5, 2.0}) {
            const int64_t n = std::max<int64_t>(1, std::min<int64_t>(slen, (int64_t)std::llround(nsb * f)));
            const int h = (int)((slen + n - 1) / n);
            if (std::find(tried.begin(), tried.end(), h) != tried.end()) continue;
            tried.push_back(h);
            if (!time_cand(Cand{w0.bt, h, w0.tile, model_for(p, w0.bt, h)})) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(b);
    if (status) {
        p->bt = save_bt;
        p->hsn = save_hsn;
        p->tile = save_tile;
        return status;
    }
    p->bt = win.bt;
    p->hsn = win.hsn;
    p->tile = win.tile;
    p->model_gcells = win.model;
    p->measured_gcells = best;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = TuneVal{win.bt, win.hsn, win.tile, win.model, best};
    }
    return ok();
}

// ---------------------------------------------------------------------------
// Allocation-free entry point (declared in an5d.h as an5d_run_noalloc).
//
// For callers that cannot call cudaMalloc: frameworks that hand all device
// memory to their own pool or caching allocator (a stray cudaMalloc can fail
// against that budget or fragment it) and loops that must not stall, since
// cudaMalloc/cudaFree may synchronise the device.  The ping-pong buffer and
// the device status word live in one file-scope device array instead of a
// plan.  Every GPU that loads this library holds the array until the process
// exits.  All calls share it: calls whose GPU work overlaps (other threads,
// other streams) race on it.

namespace {
constexpr size_t NOALLOC_HEADER = 256;  // status word at offset 0; grid buffer after it
std::mutex g_noalloc_mu;
void *g_noalloc_base[64] = {};          // device address of the array, per device
}  // namespace

static __device__ __align__(256) unsigned char an5d_noalloc_scratch[NOALLOC_HEADER +
                                                                    AN5D_NOALLOC_MAX_BYTES];

// Once per device, with that device current: the array's device address.
// (Host code must not pass the symbol itself to a kernel: on the host it is
// only a stand-in, not a device address.)
static int noalloc_base(int dev, void **out)
{
    if (dev < 0 || dev >= 64) return fail(AN5D_ERR_UNSUPPORTED, "device index %d >= 64", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, an5d_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(AN5D_ERR_CUDA, "cudaGetSymbolAddress(an5d_noalloc_scratch): %s",
                        cudaGetErrorString(e));
        g_noalloc_base[dev] = p;
    }
    *out = g_noalloc_base[dev];
    return AN5D_OK;
}

extern "C" int an5d_run_noalloc(int ndim, an5d_shape shape, int radius, const double *coeffs,
                                an5d_dtype dtype, const int64_t *dims, const void *in, void *out,
                                int64_t T, void *stream)
{
    int n = an5d_coeff_count(ndim, shape, radius);
    if (n < 0) return n;
    if (n > MAX_COEFFS)
        return fail(AN5D_ERR_UNSUPPORTED, "%d coefficients exceed the library's %d", n, MAX_COEFFS);
    if (!coeffs || !dims) return fail(AN5D_ERR_INVALID_ARG, "coeffs and dims must not be NULL");
    if (dtype < AN5D_F32 || dtype > AN5D_F32_COMPENSATED)
        return fail(AN5D_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    int64_t total = 1;
    for (int i = 0; i < ndim; ++i) {
        if (dims[i] < 1 || dims[i] > (1ll << 30))
            return fail(AN5D_ERR_INVALID_ARG, "dims[%d] = %lld out of range", i, (long long)dims[i]);
        total *= dims[i] + 2 * radius;
        if (total >= (1ll << 31))
            return fail(AN5D_ERR_UNSUPPORTED, "padded array must have fewer than 2^31 elements");
    }
    const size_t bytes = (size_t)total * elem_size(dtype);
    if (bytes > (size_t)AN5D_NOALLOC_MAX_BYTES)
        return fail(AN5D_ERR_INVALID_ARG,
                    "an5d_run_noalloc: padded grid of %zu bytes exceeds its %zu-byte limit "
                    "(use a plan and an5d_run)",
                    bytes, (size_t)AN5D_NOALLOC_MAX_BYTES);

    an5d_plan p;  // on the stack: owns nothing
    p.ndim = ndim;
    p.shape = shape;
    p.radius = radius;
    p.dtype = dtype;
    p.n = n;
    for (int i = 0; i < 3; ++i) p.dims[i] = i < ndim ? dims[i] : 0;
    p.nz = ndim == 3 ? dims[0] : 1;
    p.ny = dims[ndim - 2];
    p.nx = dims[ndim - 1];
    p.total = total;
    p.bytes = bytes;
    const bool dbl = dtype == AN5D_F64;
    for (int k = 0; k < n; ++k) p.coeffs[k] = dbl ? coeffs[k] : (double)(float)coeffs[k];
    p.bt_max = largest_bt(&p);
    if (p.bt_max == 0)
        return fail(AN5D_ERR_UNSUPPORTED, "stencil ndim=%d shape=%d R=%d dtype=%d is not built",
                    ndim, (int)shape, radius, (int)dtype);
    CUDA_TRY(cudaGetDevice(&p.device));
    CUDA_TRY(cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, p.device));
    void *base = nullptr;
    if (int s = noalloc_base(p.device, &base)) return s;
    p.d_status = static_cast<int *>(base);
    p.scratch = static_cast<unsigned char *>(base) + NOALLOC_HEADER;
    choose_default(&p);
    if (int s = check_run_args(&p, in, out, T)) return s;

    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    auto enqueue = [&]() -> int {
        CUDA_TRY(cudaMemsetAsync(p.d_status, 0, sizeof(int), st));  // the array keeps old contents
        if (T == 0) {
            CUDA_TRY(cudaMemcpyAsync(out, in, p.bytes, cudaMemcpyDeviceToDevice, st));
        } else {
            // Same pass list as an5d_run, walked without a container.
            const int64_t full = T / p.bt;
            const int rem = (int)(T % p.bt);
            const int64_t np = full + (rem ? 1 : 0);
            if (int s = launch_halo_copy(&p, in, out, st)) return s;
            if (np > 1)
                if (int s = launch_halo_copy(&p, in, p.scratch, st)) return s;
            const void *src = in;
            for (int64_t k = 0; k < np; ++k) {
                void *dst = ((np - 1 - k) % 2 == 0) ? out : p.scratch;
                if (int s = launch_pass(&p, k < full ? p.bt : rem, src, dst, st)) return s;
                src = dst;
            }
        }
        CUDA_TRY(cudaMemcpyAsync(&h, p.d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
        return AN5D_OK;
    };
    if (int s = enqueue()) {
        // work queued before the failure still uses the shared array: let it
        // finish, so that the array is idle when the call returns
        cudaStreamSynchronize(st);
        return s;
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    if (h & STATUS_TIMEOUT) return fail(AN5D_ERR_TIMEOUT, "a bounded device wait gave up");
    return ok();
}

// ---------------------------------------------------------------------------
// Internal accessors for the other translation units (adjoint).

namespace an5d {

int plan_view(const an5d_plan *p, PlanView *v)
{
    if (!p || !v) return fail(AN5D_ERR_INVALID_ARG, "NULL plan");
    v->ndim = p->ndim;
    v->shape = p->shape;
    v->radius = p->radius;
    v->dtype = p->dtype;
    v->post = p->post;
    v->n = p->n;
    v->bt = p->bt;
    v->hsn = p->hsn;
    v->tile = p->tile;
    v->device = p->device;
    v->nz = p->nz;
    v->ny = p->ny;
    v->nx = p->nx;
    v->total = p->total;
    v->bytes = p->bytes;
    v->coeffs = p->coeffs;
    return AN5D_OK;
}

int plan_fill_pass(const an5d_plan *p, int bt, int tile, const void *src, void *dst, PassDesc *d)
{
    PassGeom g;
    if (int s = pass_geometry(p, bt, p->hsn, &g, tile)) return s;
    memset(d, 0, sizeof(*d));
    const int A = 16 / (int)elem_size(p->dtype);
    if (int s = encode_row_map(&d->tmap, src, p->dtype, p->total, g.k->tile_x + A)) return s;
    d->dst = dst;
    d->status = p->d_status;
    d->pitch = p->nx + 2 * p->radius;
    d->plane = d->pitch * (p->ny + 2 * p->radius);
    d->nz = (int)p->nz;
    d->ny = (int)p->ny;
    d->nx = (int)p->nx;
    d->tile_stride_x = g.tile_stride_x;
    d->x_base = g.x_base;
    d->tile_stride_y = g.tile_stride_y;
    d->tiles_x = g.tiles_x;
    d->tiles_y = g.tiles_y;
    d->hsn = g.hsn;
    d->stream_blocks = g.stream_blocks;
    d->total_units = g.units;
    d->ctas = g.ctas;
    d->post_c = p->post_c;
    for (int k = 0; k < p->n; ++k) d->coeffs[k] = p->coeffs[k];
    return AN5D_OK;
}

int plan_launch_pass(const an5d_plan *p, int bt, const void *src, void *dst, cudaStream_t st)
{
    return launch_pass(p, bt, src, dst, st);
}

int plan_launch_halo_copy(const an5d_plan *p, const void *src, void *dst, cudaStream_t st)
{
    return launch_halo_copy(p, src, dst, st);
}

int set_error(int status, const char *msg) { return fail(status, "%s", msg); }

void *plan_work_buffer(an5d_plan *p, size_t bytes)
{
    if (p->work_bytes < bytes) {
        cudaDeviceSynchronize();  // the old buffer may still be in use by queued work
        cudaFree(p->work);
        p->work = nullptr;
        p->work_bytes = 0;
        if (cudaMalloc(&p->work, bytes) != cudaSuccess) return nullptr;
        p->work_bytes = bytes;
    }
    return p->work;
}

}  // namespace an5d

extern "C" int an5d_plan_inject_stall(an5d_plan *p, int enable)
{
    if (!p) return fail(AN5D_ERR_INVALID_ARG, "NULL plan");
    if (p->ndim != 2) return fail(AN5D_ERR_UNSUPPORTED, "stall injection is built for 2D plans");
    p->stall_test = enable ? 1 : 0;
    return ok();
}
