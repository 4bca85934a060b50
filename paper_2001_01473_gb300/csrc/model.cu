// model.cu -- analytic roofline model of the streamed sweep kernels and the
// microbenchmarks that measure its peaks (copy, FP32/FP64 fma, shared-memory
// loads), as the paper measures its own peaks before modelling (Section 4:
// global and shared memory peaks from micro-benchmarks, compute from the
// FMA rate with an ALU-efficiency factor).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "an5d.h"
#include "an5d_internal.h"
#include "device_common.cuh"
#include "model.h"

namespace an5d {

static std::mutex g_peaks_mu;
static Peaks g_measured[64];

static Peaks nominal_peaks(int dev)
{
    Peaks p;
    int sms = 0, clk = 0, mclk = 0, bus = 0, ratio = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    cudaDeviceGetAttribute(&mclk, cudaDevAttrMemoryClockRate, dev);
    cudaDeviceGetAttribute(&bus, cudaDevAttrGlobalMemoryBusWidth, dev);
    cudaDeviceGetAttribute(&ratio, cudaDevAttrSingleToDoublePrecisionPerfRatio, dev);
    p.sms = sms;
    p.sm_clock_mhz = clk / 1e3;
    p.hbm_gbs = 2.0 * mclk * 1e3 * (bus / 8.0) / 1e9;
    p.fp32_gflops = sms * 128.0 * 2.0 * clk * 1e3 / 1e9;
    p.fp64_gflops = ratio > 0 ? p.fp32_gflops / ratio : p.fp32_gflops / 64.0;
    p.smem_gbs = sms * 128.0 * clk * 1e3 / 1e9;
    p.measured = 0;
    return p;
}

Peaks current_peaks()
{
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_peaks_mu);
        if (dev >= 0 && dev < 64 && g_measured[dev].measured) return g_measured[dev];
    }
    return nominal_peaks(dev);
}

// Warp instructions issued per warp per streaming iteration (one input row).
static double warp_instr_per_iter(const ModelInput &m, double n_terms, double cells_per_lane)
{
    const double V = cells_per_lane;
    const double R = m.radius;
    double per_term = 1.0;                      // one fma / mul per cell and term
    if (m.dtype == DT_F32C) per_term = 10.0;    // Dot2: TwoProduct + TwoSum + 2 adds
    const double shuffles = 2.0 * R * (m.dtype == DT_F64 ? 2.0 : 1.0);
    const double cvt = m.dtype == DT_F16S ? 2.0 * V : 0.0;
    const double level = V * n_terms * per_term + shuffles + cvt + 2.0;
    return m.bt * level + 3.0 * V + 12.0;       // + row load, store, ring/barrier bookkeeping
}

double model_gcells(const ModelInput &m)
{
    const Peaks pk = current_peaks();
    if (pk.sms <= 0 || m.units <= 0) return 0.0;
    const double w = m.dtype == DT_F64 ? 8.0 : (m.dtype == DT_F16S ? 2.0 : 4.0);
    const double R = m.radius;
    double n = 0;
    if (m.ndim == 2) n = m.shape == SH_STAR ? 4 * R + 1 : (2 * R + 1) * (2 * R + 1);
    else n = m.shape == SH_STAR ? 6 * R + 1 : (2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    const double cells = (double)m.nz * m.ny * m.nx;
    const double useful = cells * m.bt;  // cell-updates per pass

    // Streaming iterations per unit: its stream block plus the bT*R lead-in
    // and lead-out rows (Section 3.2's redundant sub-planes).
    const double iters = m.hsn + 2.0 * m.bt * R;
    double hbm_bytes, warp_instr, fma_lanes;
    // cells per lane of the kernel: 2D tiles are one warp wide
    const double V = m.ndim == 2 ? m.tile_x / 32.0 : CELLS_PER_LANE;
    if (m.ndim == 2) {
        const double rowbuf = m.tile_x + 16.0 / w;
        hbm_bytes = (double)m.units * iters * rowbuf * w + cells * w;
        warp_instr = (double)m.units * iters * warp_instr_per_iter(m, n, V);
        fma_lanes = (double)m.units * iters * m.bt * 32.0 * V * n *
                    (m.dtype == DT_F32C ? 3.0 : 1.0);
    } else {
        const double plane = (double)m.tile_x * m.tile_y;
        hbm_bytes = (double)m.units * iters * plane * w + cells * w;
        const double warps = plane / (32.0 * V);
        warp_instr = (double)m.units * iters * warps * warp_instr_per_iter(m, n, V);
        fma_lanes = (double)m.units * iters * m.bt * plane * n * (m.dtype == DT_F32C ? 3.0 : 1.0);
    }
    const double clk = pk.sm_clock_mhz * 1e6;
    const double t_hbm = hbm_bytes / (pk.hbm_gbs * 1e9);
    const double t_issue = warp_instr / (pk.sms * 4.0 * clk);
    const double fma_rate = (m.dtype == DT_F64 ? pk.fp64_gflops : pk.fp32_gflops) * 1e9 / 2.0;
    const double t_fma = fma_lanes / fma_rate;
    const double waves = std::ceil((double)m.units / std::max(1, m.resident_units));
    const double eff_sm = (double)m.units / (waves * std::max(1, m.resident_units));
    const double t = std::max(t_hbm, std::max(t_issue, t_fma)) / std::max(eff_sm, 1e-3);
    return useful / t / 1e9;
}

// ---------------------------------------------------------------------------
// Microbenchmarks.

__global__ void mb_copy(const float4 *__restrict__ a, float4 *__restrict__ b, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

template <typename T>
__global__ void mb_fma(T *out, int iters, T seed)
{
    T a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    T a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    const T m = (T)0.999999, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            a0 = op_fma(a0, m, c); a1 = op_fma(a1, m, c); a2 = op_fma(a2, m, c); a3 = op_fma(a3, m, c);
            a4 = op_fma(a4, m, c); a5 = op_fma(a5, m, c); a6 = op_fma(a6, m, c); a7 = op_fma(a7, m, c);
        }
    }
    const T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == (T)-12345.0) out[threadIdx.x] = s;  // keeps the chains alive
}

__global__ void mb_smem(unsigned *out, int iters)
{
    __shared__ uint4 buf[1024];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x)
        buf[i] = make_uint4(i, i * 3u, i * 5u, i * 7u);
    __syncthreads();
    uint4 acc = make_uint4(0, 0, 0, 0);
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint4 v = buf[(idx + u * 128) & 1023];
            acc.x ^= v.x; acc.y ^= v.y; acc.z ^= v.z; acc.w ^= v.w;
        }
        idx += 32;
    }
    if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x9e3779b9u) out[threadIdx.x] = acc.x;
}

}  // namespace an5d

using namespace an5d;

static void to_c(const Peaks &p, an5d_peaks *o)
{
    o->hbm_gbs = p.hbm_gbs;
    o->fp32_gflops = p.fp32_gflops;
    o->fp64_gflops = p.fp64_gflops;
    o->smem_gbs = p.smem_gbs;
    o->sm_clock_mhz = p.sm_clock_mhz;
    o->sms = p.sms;
    o->measured = p.measured;
}

extern "C" int an5d_get_peaks(an5d_peaks *out)
{
    if (!out) return AN5D_ERR_INVALID_ARG;
    to_c(current_peaks(), out);
    return AN5D_OK;
}

extern "C" int an5d_measure_peaks(an5d_peaks *out, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return AN5D_ERR_CUDA;
    Peaks p = nominal_peaks(dev);
    const size_t bytes = 1ull << 30;  // 1 GiB per buffer: well above the L2
    void *a = nullptr, *b = nullptr, *o = nullptr;
    if (cudaMalloc(&a, bytes) != cudaSuccess) return AN5D_ERR_OOM;
    if (cudaMalloc(&b, bytes) != cudaSuccess) { cudaFree(a); return AN5D_ERR_OOM; }
    if (cudaMalloc(&o, 4096 * sizeof(double)) != cudaSuccess) { cudaFree(a); cudaFree(b); return AN5D_ERR_OOM; }
    cudaMemsetAsync(a, 0, bytes, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](auto &&launch, int reps) {
        launch();
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms * 1e-3 / reps;
    };
    const size_t n4 = bytes / sizeof(float4);
    const int blocks = p.sms * 8;
    double t = timed([&] { mb_copy<<<blocks, 256, 0, st>>>((const float4 *)a, (float4 *)b, n4); }, 10);
    p.hbm_gbs = 2.0 * bytes / t / 1e9;
    const int iters = 4096;
    t = timed([&] { mb_fma<float><<<p.sms * 8, 256, 0, st>>>((float *)o, iters, 1.0f); }, 5);
    p.fp32_gflops = 2.0 * 8 * 16 * (double)iters * p.sms * 8 * 256 / t / 1e9;
    const int diters = 256;
    t = timed([&] { mb_fma<double><<<p.sms * 8, 256, 0, st>>>((double *)o, diters, 1.0); }, 3);
    p.fp64_gflops = 2.0 * 8 * 16 * (double)diters * p.sms * 8 * 256 / t / 1e9;
    const int siters = 8192;
    t = timed([&] { mb_smem<<<p.sms * 8, 128, 0, st>>>((unsigned *)o, siters); }, 5);
    p.smem_gbs = 16.0 * 8 * (double)siters * p.sms * 8 * 128 / t / 1e9;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(b);
    cudaFree(o);
    if (cudaGetLastError() != cudaSuccess) return AN5D_ERR_CUDA;
    p.measured = 1;
    {
        std::lock_guard<std::mutex> lk(g_peaks_mu);
        g_measured[dev] = p;
    }
    if (out) to_c(p, out);
    return AN5D_OK;
}
