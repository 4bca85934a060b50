// adjoint.cu -- adjoint (reverse-mode gradient) of the FP32 plain method.
//
// For a loss L(u_T) the caller supplies g_T = dL/du_T; the library returns
// dL/du_0 (interior; the halo is boundary data, not a parameter) and
// dL/dc_k.  With S the one-step operator restricted to the interior:
//     g_t = S^T g_{t+1}                  (transposed stencil: offsets -o_k,
//                                         zero Dirichlet halo)
//     dL/dc_k = sum_t sum_{p interior} g_{t+1}[p] * u_t[p + o_k]
// (the paper has no adjoint; this follows from differentiating the time loop
// of Section 3.3 / Fig. 5).
//
// Schedule (checkpointing with recomputation inside each block of bT steps):
//   forward: N.5D-blocked passes of degree bT keep u_{m bT} as checkpoints;
//   backward, block m (steps t0 .. t0+nb-1), last block first:
//     1. one blocked pass of degree nb-1 from the checkpoint recomputes and
//        stores u_{t0+1} .. u_{t0+nb-1};
//     2. one blocked pass of degree nb of the transposed stencil takes
//        g_{t0+nb} to g_{t0}, storing every level;
//     3. dL/dc_k += <g_{t+1}, shift_k u_t> for the nb steps of the block
//        (FP32 per thread over a fixed partition, FP64 across threads).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "an5d.h"
#include "an5d_internal.h"
#include "sweep2d.cuh"

namespace an5d {

constexpr int ADJ_MAX_BT = 4;

struct LevelPtrs {
    float *p[ADJ_MAX_BT + 1];  // p[t] receives level t, t = 1..bT-1
};

template <int SHAPE, int R, int BT>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32, (Sweep2DOccupancy<float, SHAPE, BT, R, MODE_PLAIN>::value))
    sweep2d_levels_kernel(const __grid_constant__ CUtensorMap tmap,
                          const Sweep2DArgs<float, NCoeff2<SHAPE, R>::value> a, const LevelPtrs lv)
{
    using G = Sweep2DGeom<float, BT, R>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * WARPS_PER_CTA + warp;
    if (gw >= a.total_warps) return;
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
    tg.stall = 0;
    unsigned char *const smem_al = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    sweep2d_tile<SHAPE, R, BT, float, MODE_PLAIN, false, decltype(a.k.c), decltype(a.k.c), true>(
        tg, &tmap, a.dst, a.status, smem_al + warp * G::WARP_BYTES, a.k.c, a.k.c, lv.p);
}

// Canonical offset k of a 2D stencil (star: centre, then (dx=i), (dy=i) for
// i = -R..-1, 1..R; box: dy outer, dx inner).
template <int SHAPE, int R> __host__ __device__ constexpr int off_dy(int k)
{
    if (SHAPE == SH_BOX) return k / (2 * R + 1) - R;
    if (k == 0) return 0;
    const int j = (k - 1) / 2, i = j < R ? j - R : j - R + 1;
    return (k - 1) % 2 == 1 ? i : 0;
}
template <int SHAPE, int R> __host__ __device__ constexpr int off_dx(int k)
{
    if (SHAPE == SH_BOX) return k % (2 * R + 1) - R;
    if (k == 0) return 0;
    const int j = (k - 1) / 2, i = j < R ? j - R : j - R + 1;
    return (k - 1) % 2 == 0 ? i : 0;
}

constexpr int CORR_BLOCKS = 2048;  // at most; a grid uses corr_blocks(ny, nx) of them
constexpr int CORR_THREADS = 256;

// Fixed partition of a grid for the coefficient reduction: column groups of
// CORR_THREADS columns times bands of about 64 rows, at most CORR_BLOCKS
// blocks.  Depends only on the grid, so the reduction order is fixed.
__host__ __device__ inline void corr_split(int ny, int nx, int *ncx, int *nby)
{
    int cx = (nx + CORR_THREADS - 1) / CORR_THREADS;
    if (cx > CORR_BLOCKS) cx = CORR_BLOCKS;
    int by = (ny + 63) / 64;
    if (by > CORR_BLOCKS / cx) by = CORR_BLOCKS / cx;
    *ncx = cx;
    *nby = by < 1 ? 1 : by;
}
__host__ __device__ inline int corr_blocks(int ny, int nx)
{
    int cx, by;
    corr_split(ny, nx, &cx, &by);
    return cx * by;
}

// part[b * n + k] += sum over block b's cells of g[p] * u[p + o_k] (interior
// p).  Block b owns a band of rows of a column group; each thread walks down
// its columns keeping the (2R+1) x (2R+1) neighbourhood of u in registers (a
// ring of rows indexed by row mod 2R+1, so every index is static), which
// reads 2R+2 values per cell instead of one per offset.  Each block owns its
// slots and launches on one stream are ordered: the accumulation over steps
// is deterministic.
// The (g_{t+1}, u_t) pairs of the steps of one block.
struct CorrSteps {
    const float *g[ADJ_MAX_BT];
    const float *u[ADJ_MAX_BT];
    int n;
};

template <int SHAPE, int R>
__global__ void __launch_bounds__(CORR_THREADS)
    corr_kernel(const CorrSteps steps, int ny, int nx, double *part)
{
    constexpr int N = NCoeff2<SHAPE, R>::value;
    constexpr int P = 2 * R + 1;
    const int pitch = nx + 2 * R;
    int ncx, nby;
    corr_split(ny, nx, &ncx, &nby);
    const int cx = blockIdx.x % ncx, by = blockIdx.x / ncx;
    // bands start on multiples of P, so the ring slot of row y is (y - y0) mod P
    const int rpb = ((ny + nby - 1) / nby + P - 1) / P * P;
    const int y0 = by * rpb, y1 = min(ny, y0 + rpb);
    constexpr int NWARP = CORR_THREADS / 32;
    __shared__ double wsum[NWARP][N];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int step = 0; step < steps.n; ++step) {
    const float *__restrict__ g = steps.g[step];
    const float *__restrict__ u = steps.u[step];
    float acc[N];
#pragma unroll
    for (int k = 0; k < N; ++k) acc[k] = 0.f;
    for (int x = cx * CORR_THREADS + threadIdx.x; x < nx && y0 < y1; x += ncx * CORR_THREADS) {
        // w[s][j]: u at interior row y0 + m (m mod P = s) and column x + j - R
        const float *ucol = u + R + x;                        // padded column x + R
        const float *gcol = g + (int64_t)R * pitch + R + x;   // interior cell (0, x)
        float w[P][P];
#pragma unroll
        for (int d = 0; d < 2 * R; ++d) {                     // rows y0 - R .. y0 + R - 1
            const float *row = ucol + (int64_t)(y0 + d) * pitch;
#pragma unroll
            for (int j = 0; j < P; ++j) w[((d - R) % P + P) % P][j] = row[j - R];
        }
        for (int yb = y0; yb < y1; yb += P) {
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int y = yb + q;
                if (y < y1) {
                    const float *row = ucol + (int64_t)(y + 2 * R) * pitch;   // row y + R
#pragma unroll
                    for (int j = 0; j < P; ++j) w[(q + R) % P][j] = row[j - R];
                    const float gv = gcol[(int64_t)y * pitch];
#pragma unroll
                    for (int k = 0; k < N; ++k) {
                        const int dy = off_dy<SHAPE, R>(k), dx = off_dx<SHAPE, R>(k);
                        acc[k] = __fmaf_rn(gv, w[((q + dy) % P + P) % P][dx + R], acc[k]);
                    }
                }
            }
        }
    }
    // FP64 reduction in a fixed order, per step: a shuffle tree inside each
    // warp, then the warps' sums in warp order (acc stays in registers:
    // every index is static)
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double v = (double)acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL_MASK, v, o);
        if (lane == 0) wsum[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < NWARP; ++w) v += wsum[w][threadIdx.x];
        part[blockIdx.x * N + threadIdx.x] += v;
    }
    __syncthreads();  // wsum is reused by the next step
    }
}

// dc[k] = sum_b part[b * n + k]: one block per coefficient, a fixed strided
// split over its threads and a fixed tree (deterministic).
__global__ void __launch_bounds__(CORR_THREADS) corr_final(const double *__restrict__ part, int n, int blocks, double *dc)
{
    const int k = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < blocks; b += CORR_THREADS) s += part[b * n + k];
    __shared__ double red[CORR_THREADS];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = CORR_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) dc[k] = red[0];
}

// dst := src on the interior, 0 on the halo.
__global__ void interior_copy_kernel(const float *__restrict__ src, float *__restrict__ dst, int ny, int nx, int R)
{
    const int pitch = nx + 2 * R;
    const int64_t total = (int64_t)(ny + 2 * R) * pitch;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(q / pitch), x = (int)(q % pitch);
        dst[q] = (y >= R && y < ny + R && x >= R && x < nx + R) ? src[q] : 0.f;
    }
}

}  // namespace an5d

// ---------------------------------------------------------------------------
// Host driver.

using namespace an5d;

namespace {

using LevelsLaunch = cudaError_t (*)(const PassDesc &, const LevelPtrs &, cudaStream_t);
using CorrLaunch = void (*)(const CorrSteps &, int, int, double *, cudaStream_t);

template <int SHAPE, int R, int BT>
cudaError_t launch_levels(const PassDesc &d, const LevelPtrs &lv, cudaStream_t st)
{
    constexpr int N = NCoeff2<SHAPE, R>::value;
    using G = Sweep2DGeom<float, BT, R>;
    // the descriptor must describe this kernel's tile width (its TMA box too)
    if (d.tile_stride_x != G::TILE - 2 * BT * R) return cudaErrorInvalidValue;
    Sweep2DArgs<float, N> a;
    a.dst = static_cast<float *>(d.dst);
    a.status = d.status;
    a.pitch = static_cast<int>(d.pitch);
    a.ny = d.ny;
    a.nx = d.nx;
    a.tile_stride = d.tile_stride_x;
    a.xb0 = d.x_base;
    a.tiles_x = d.tiles_x;
    a.hsn = d.hsn;
    a.total_warps = d.total_units;
    a.stall_test = 0;
    for (int k = 0; k < N; ++k) {
        a.k.c[k] = static_cast<float>(d.coeffs[k]);
        a.kp.c[k] = 0;
    }
    auto fn = sweep2d_levels_kernel<SHAPE, R, BT>;
    if (G::CTA_BYTES > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::CTA_BYTES);
        if (e != cudaSuccess) return e;
    }
    fn<<<d.ctas, WARPS_PER_CTA * 32, G::CTA_BYTES, st>>>(d.tmap, a, lv);
    return cudaGetLastError();
}

template <int SHAPE, int R>
void launch_corr(const CorrSteps &steps, int ny, int nx, double *part, cudaStream_t st)
{
    corr_kernel<SHAPE, R><<<corr_blocks(ny, nx), CORR_THREADS, 0, st>>>(steps, ny, nx, part);
}

template <int SHAPE, int R> LevelsLaunch levels_for(int bt)
{
    switch (bt) {
    case 1: return &launch_levels<SHAPE, R, 1>;
    case 2: return &launch_levels<SHAPE, R, 2>;
    case 3: return &launch_levels<SHAPE, R, 3>;
    default: return &launch_levels<SHAPE, R, 4>;
    }
}

LevelsLaunch find_levels(int shape, int R, int bt)
{
    if (shape == SH_STAR) return R == 1 ? levels_for<SH_STAR, 1>(bt) : levels_for<SH_STAR, 2>(bt);
    return R == 1 ? levels_for<SH_BOX, 1>(bt) : levels_for<SH_BOX, 2>(bt);
}

CorrLaunch find_corr(int shape, int R)
{
    if (shape == SH_STAR) return R == 1 ? &launch_corr<SH_STAR, 1> : &launch_corr<SH_STAR, 2>;
    return R == 1 ? &launch_corr<SH_BOX, 1> : &launch_corr<SH_BOX, 2>;
}

// Index of the mirrored offset -o_k in the canonical order.
int mirror_index(int shape, int R, int k)
{
    if (shape == SH_BOX) return (2 * R + 1) * (2 * R + 1) - 1 - k;
    if (k == 0) return 0;
    // star: k-1 = 2*j + (0: dx, 1: dy), j over i = -R..-1, 1..R; -i is j' = 2R-1-j
    const int j = (k - 1) / 2, axis = (k - 1) % 2;
    return 1 + 2 * (2 * R - 1 - j) + axis;
}

}  // namespace

extern "C" int an5d_run_adjoint(an5d_plan *plan, const void *u0, const void *gT, void *grad_u0,
                                double *grad_coeffs, int64_t T, void *stream)
{
    PlanView v;
    if (int s = plan_view(plan, &v)) return s;
    if (v.ndim != 2 || v.dtype != AN5D_F32 || v.radius > 2 || v.post != POST_NONE)
        return set_error(AN5D_ERR_UNSUPPORTED,
                         "adjoint: 2D FP32 plans of radius 1-2 without a per-step division only");
    if (!u0 || !gT || !grad_u0 || !grad_coeffs || T < 0)
        return set_error(AN5D_ERR_INVALID_ARG, "adjoint: NULL argument or T < 0");
    if ((((uintptr_t)u0) | ((uintptr_t)gT) | ((uintptr_t)grad_u0)) & 15)
        return set_error(AN5D_ERR_INVALID_ARG, "adjoint: buffers must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const int R = v.radius, n = v.n;
    const int ny = (int)v.ny, nx = (int)v.nx;
    const int bt = std::max(1, std::min(v.bt, ADJ_MAX_BT));
    const int64_t M = (T + bt - 1) / bt;
    // one work allocation, owned and reused by the plan: checkpoints C[1..M-1],
    // u levels U[1..bt-1], g levels G[0..bt], dc and the reduction partials
    const size_t gbytes = (v.bytes + 255) / 256 * 256;
    const size_t ngrids = (size_t)std::max<int64_t>(M - 1, 0) + (bt - 1) + (bt + 1);
    char *work = static_cast<char *>(
        plan_work_buffer(plan, ngrids * gbytes + sizeof(double) * (n + (size_t)CORR_BLOCKS * n)));
    if (!work) return set_error(AN5D_ERR_OOM, "adjoint: work memory");
    size_t next = 0;
    auto grid = [&]() -> void * {
        void *p = work + next;
        next += gbytes;
        return p;
    };
    double *dc = reinterpret_cast<double *>(work + ngrids * gbytes);
    double *part = dc + n;
    cudaMemsetAsync(dc, 0, sizeof(double) * (n + (size_t)CORR_BLOCKS * n), st);
    std::vector<double> mc(n);
    for (int k = 0; k < n; ++k) mc[k] = v.coeffs[mirror_index(v.shape, R, k)];

    // gradient of the final state, zero on the halo
    std::vector<void *> G(bt + 1);
    for (int j = 0; j <= bt; ++j) {
        G[j] = grid();
        cudaMemsetAsync(G[j], 0, v.bytes, st);
    }
    interior_copy_kernel<<<1024, 256, 0, st>>>((const float *)gT, (float *)G[0], ny, nx, R);
    if (M == 0) {
        cudaMemcpyAsync(grad_u0, G[0], v.bytes, cudaMemcpyDeviceToDevice, st);
        for (int k = 0; k < n; ++k) grad_coeffs[k] = 0.0;
        return cudaStreamSynchronize(st) == cudaSuccess ? AN5D_OK : set_error(AN5D_ERR_CUDA, "sync");
    }

    // forward: checkpoints C[m] = u_{m bt}, m = 0..M-1 (C[0] = u0)
    std::vector<const void *> C(M);
    C[0] = u0;
    for (int64_t m = 1; m < M; ++m) {
        void *b = grid();
        if (int s = plan_launch_halo_copy(plan, u0, b, st)) return s;
        if (int s = plan_launch_pass(plan, bt, C[m - 1], b, st)) return s;
        C[m] = b;
    }
    std::vector<void *> U(bt);
    for (int s2 = 1; s2 < bt; ++s2) {
        U[s2] = grid();
        if (int s = plan_launch_halo_copy(plan, u0, U[s2], st)) return s;
    }
    CorrLaunch corr = find_corr(v.shape, R);

    // backward, last block first
    for (int64_t m = M - 1; m >= 0; --m) {
        const int nb = (int)std::min<int64_t>(bt, T - m * bt);
        // 1. recompute u_{t0+1} .. u_{t0+nb-1} from the checkpoint
        if (nb >= 2) {
            PassDesc d;
            if (int s = plan_fill_pass(plan, nb - 1, 0, C[m], U[nb - 1], &d)) return s;
            LevelPtrs lv = {};
            for (int t = 1; t < nb - 1; ++t) lv.p[t] = (float *)U[t];
            cudaError_t e = find_levels(v.shape, R, nb - 1)(d, lv, st);
            if (e != cudaSuccess) return set_error(AN5D_ERR_CUDA, cudaGetErrorString(e));
        }
        // 2. transposed stencil: g_{t0+nb} -> g_{t0}, every level stored (G[j] = g_{t0+nb-j})
        {
            PassDesc d;
            if (int s = plan_fill_pass(plan, nb, 0, G[0], G[nb], &d)) return s;
            for (int k = 0; k < n; ++k) d.coeffs[k] = mc[k];
            LevelPtrs lv = {};
            for (int t = 1; t < nb; ++t) lv.p[t] = (float *)G[t];
            cudaError_t e = find_levels(v.shape, R, nb)(d, lv, st);
            if (e != cudaSuccess) return set_error(AN5D_ERR_CUDA, cudaGetErrorString(e));
        }
        // 3. dL/dc += <g_{t+1}, shift_k u_t> for t = t0 .. t0+nb-1 (one launch)
        {
            CorrSteps cs = {};
            cs.n = nb;
            for (int s2 = 0; s2 < nb; ++s2) {
                cs.g[s2] = (const float *)G[nb - 1 - s2];
                cs.u[s2] = (const float *)(s2 == 0 ? C[m] : U[s2]);
            }
            corr(cs, ny, nx, part, st);
        }
        std::swap(G[0], G[nb]);
    }
    corr_final<<<n, CORR_THREADS, 0, st>>>(part, n, corr_blocks(ny, nx), dc);
    cudaMemcpyAsync(grad_u0, G[0], v.bytes, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(grad_coeffs, dc, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(AN5D_ERR_CUDA, cudaGetErrorString(e));
    return an5d_plan_status(plan);
}
