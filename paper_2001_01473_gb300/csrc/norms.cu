// norms.cu -- FP64 error norms of a run against an FP64 reference grid.
//
// The precision forms (binary16 storage, Dot2-compensated FP32) are measured
// by their distance from an FP64 evaluation of the same sweep: the maximum
// absolute difference and the L2 norms over the interior.  Sums run in FP64
// over a fixed partition (1024 blocks, fixed tree inside a block, one
// block for the final combine), so a given grid always gives the same bits.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "an5d.h"
#include "an5d_internal.h"

namespace an5d {

constexpr int NORM_BLOCKS = 1024;
constexpr int NORM_THREADS = 256;

template <typename S> __device__ __forceinline__ double to_d(S v) { return (double)v; }
template <> __device__ __forceinline__ double to_d<__half>(__half v) { return (double)__half2float(v); }

// Partial norms of interior rows [rb, re) (rows of the padded (z, y) index).
template <typename S>
__global__ void __launch_bounds__(NORM_THREADS)
    norms_partial(const S *__restrict__ u, const double *__restrict__ ref, int64_t rows, int nyp,
                  int nxp, int hz, int nzp, int R, double *__restrict__ part)
{
    __shared__ double smax[NORM_THREADS], sd2[NORM_THREADS], sr2[NORM_THREADS];
    const int64_t per = (rows + NORM_BLOCKS - 1) / NORM_BLOCKS;
    const int64_t rb = blockIdx.x * per, re = min(rows, rb + per);
    double m = 0.0, d2 = 0.0, r2 = 0.0;
    for (int64_t row = rb; row < re; ++row) {
        const int64_t z = row / nyp, y = row % nyp;
        if (z < hz || z >= nzp - hz || y < R || y >= nyp - R) continue;  // halo row
        const int64_t base = row * nxp;
        for (int x = R + threadIdx.x; x < nxp - R; x += NORM_THREADS) {
            const double a = to_d<S>(u[base + x]);
            const double b = ref[base + x];
            const double d = a - b;
            m = fmax(m, fabs(d));
            d2 = fma(d, d, d2);
            r2 = fma(b, b, r2);
        }
    }
    smax[threadIdx.x] = m;
    sd2[threadIdx.x] = d2;
    sr2[threadIdx.x] = r2;
    __syncthreads();
    for (int s = NORM_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
            sd2[threadIdx.x] += sd2[threadIdx.x + s];
            sr2[threadIdx.x] += sr2[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = smax[0];
        part[3 * blockIdx.x + 1] = sd2[0];
        part[3 * blockIdx.x + 2] = sr2[0];
    }
}

__global__ void __launch_bounds__(NORM_THREADS) norms_final(const double *__restrict__ part, double *__restrict__ out)
{
    __shared__ double smax[NORM_THREADS], sd2[NORM_THREADS], sr2[NORM_THREADS];
    double m = 0.0, d2 = 0.0, r2 = 0.0;
    for (int b = threadIdx.x; b < NORM_BLOCKS; b += NORM_THREADS) {
        m = fmax(m, part[3 * b]);
        d2 += part[3 * b + 1];
        r2 += part[3 * b + 2];
    }
    smax[threadIdx.x] = m;
    sd2[threadIdx.x] = d2;
    sr2[threadIdx.x] = r2;
    __syncthreads();
    for (int s = NORM_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
            sd2[threadIdx.x] += sd2[threadIdx.x + s];
            sr2[threadIdx.x] += sr2[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = smax[0];
        out[1] = sd2[0];
        out[2] = sr2[0];
    }
}

}  // namespace an5d

using namespace an5d;

extern "C" int an5d_error_norms(int ndim, int radius, const int64_t *dims, an5d_dtype dtype,
                                const void *u, const double *ref, double *out, void *stream)
{
    if ((ndim != 2 && ndim != 3) || radius < 1 || !dims || !u || !ref || !out)
        return AN5D_ERR_INVALID_ARG;
    int64_t nz = ndim == 3 ? dims[0] : 1, ny = dims[ndim - 2], nx = dims[ndim - 1];
    if (nz < 1 || ny < 1 || nx < 1) return AN5D_ERR_INVALID_ARG;
    const int hz = ndim == 3 ? radius : 0;
    const int64_t nzp = nz + 2 * hz, nyp = ny + 2 * radius, nxp = nx + 2 * radius;
    cudaStream_t st = (cudaStream_t)stream;
    double *part = nullptr, *dout = nullptr;
    if (cudaMalloc(&part, sizeof(double) * (3 * NORM_BLOCKS + 3)) != cudaSuccess) return AN5D_ERR_OOM;
    dout = part + 3 * NORM_BLOCKS;
    const int64_t rows = nzp * nyp;
    switch (dtype) {
    case AN5D_F64:
        norms_partial<double><<<NORM_BLOCKS, NORM_THREADS, 0, st>>>((const double *)u, ref, rows, (int)nyp,
                                                                   (int)nxp, hz, (int)nzp, radius, part);
        break;
    case AN5D_F16S_F32C:
        norms_partial<__half><<<NORM_BLOCKS, NORM_THREADS, 0, st>>>((const __half *)u, ref, rows, (int)nyp,
                                                                   (int)nxp, hz, (int)nzp, radius, part);
        break;
    default:
        norms_partial<float><<<NORM_BLOCKS, NORM_THREADS, 0, st>>>((const float *)u, ref, rows, (int)nyp,
                                                                  (int)nxp, hz, (int)nzp, radius, part);
    }
    norms_final<<<1, NORM_THREADS, 0, st>>>(part, dout);
    cudaError_t e = cudaMemcpyAsync(out, dout, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(part);
    return e == cudaSuccess ? AN5D_OK : AN5D_ERR_CUDA;
}
