// an5d_internal.h -- types shared by the C-ABI layer and the kernel
// translation units: launch descriptors and the kernel registry.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace an5d {

enum Dtype : int { DT_F32 = 0, DT_F64 = 1, DT_F16S = 2, DT_F32C = 3 };
enum Shape : int { SH_STAR = 0, SH_BOX = 1 };
// Per-step operation after the weighted sum (division-type stencils of Table 4):
// none, an IEEE division by the divisor, or a product with its rounded reciprocal.
enum Post : int { POST_NONE = 0, POST_DIV = 1, POST_MUL = 2 };

constexpr int MAX_COEFFS = 729;  // (2R+1)^3 for the largest stencil, box3d radius 4

// Bits of a plan's device status word.
enum : int { STATUS_TIMEOUT = 1 };
constexpr int WARPS_PER_CTA = 4;
constexpr int CELLS_PER_LANE = 4;  // consecutive x cells owned by one lane
constexpr int PREFETCH_ROWS = 3;   // TMA rows in flight ahead of the consumer

// One pass of a streamed sweep (bT fused steps) over one grid.
struct PassDesc {
    CUtensorMap tmap;        // 1D tiled map over the whole padded source array
    void *dst;               // padded destination array
    int *status;             // device status word of the plan
    int64_t pitch;           // elements per padded x row
    int64_t plane;           // elements per padded xy plane (3D)
    int nz, ny, nx;          // interior extents (nz = 1 in 2D)
    int tile_stride_x;       // output columns per tile along x
    int x_base;              // 3D: padded column where tile column 0's compute region starts
    int tile_stride_y;       // 3D: output rows per tile along y
    int tiles_x, tiles_y;    // tiles per axis
    int hsn;                 // output rows (2D) / planes (3D) per stream block
    int stream_blocks;
    int total_units;         // warps (2D) or CTAs (3D) that carry work
    int ctas;                // grid size
    int stall_test;          // fault injection (tests only)
    double post_c;           // divisor (POST_DIV) or reciprocal (POST_MUL), in the dtype's precision
    double coeffs[MAX_COEFFS];
};

using LaunchFn = cudaError_t (*)(const PassDesc &, cudaStream_t);

struct KernelKey {
    int ndim, shape, radius, dtype, bt;
    int post = POST_NONE;
    int tile = 0;  // tile variant: 0 = the default kernel, else its tile width along x
    int part = 0;  // 0 = a pass's kernel; 1 = the narrow kernel of a 3D pass's last tile column
    bool operator==(const KernelKey &o) const
    {
        return ndim == o.ndim && shape == o.shape && radius == o.radius && dtype == o.dtype &&
               bt == o.bt && post == o.post && tile == o.tile && part == o.part;
    }
};

struct KernelEntry {
    KernelKey key;
    LaunchFn launch;
    const void *func;       // for cudaFuncGetAttributes / occupancy queries
    int threads;            // threads per CTA
    size_t smem_bytes;      // dynamic shared memory per CTA
    int tile_x;             // tile width along x, overlap included
    int tile_y;             // 3D tile height along y, overlap included (1 in 2D)
    int units_per_cta;      // work units per CTA (warps in 2D, 1 in 3D)
};

std::vector<KernelEntry> &registry();

struct Registrar {
    Registrar(const KernelEntry *entries, int n)
    {
        for (int i = 0; i < n; ++i) registry().push_back(entries[i]);
    }
};

const KernelEntry *find_kernel(const KernelKey &k);

}  // namespace an5d

struct an5d_plan;

namespace an5d {

// Read-only view of a plan for translation units other than the C-ABI one.
struct PlanView {
    int ndim, shape, radius, dtype, n, bt, hsn, device;
    int tile;              // tile variant of the chosen kernel (0 = default)
    int post;              // POST_NONE unless the plan is a division-type stencil
    int64_t nz, ny, nx, total;
    size_t bytes;
    const double *coeffs;  // rounded to the compute precision
};
int plan_view(const an5d_plan *p, PlanView *v);
// Pass descriptor (tensor map over src, geometry, coefficients) of degree bt
// for the kernels of tile variant `tile` (0 = default width, -1 = the plan's
// own choice).  A caller that launches its own kernels with it must ask for
// the width those kernels are built for.
int plan_fill_pass(const an5d_plan *p, int bt, int tile, const void *src, void *dst, PassDesc *d);
int plan_launch_pass(const an5d_plan *p, int bt, const void *src, void *dst, cudaStream_t st);
int plan_launch_halo_copy(const an5d_plan *p, const void *src, void *dst, cudaStream_t st);
int set_error(int status, const char *msg);
// The plan's reusable work memory, at least `bytes` (grown on demand, owned by the plan).
void *plan_work_buffer(an5d_plan *p, size_t bytes);

}  // namespace an5d
