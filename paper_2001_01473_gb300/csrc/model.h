// model.h -- this library's analytic roofline model of one streamed pass.
//
// The paper ranks configurations with a roofline over compute, shared memory
// and global memory divided by an SM-efficiency factor (Section 4).  This
// model keeps that structure but counts what the GB300 kernels execute:
// HBM bytes moved by the TMA row loads and the stores (overlap included),
// warp instructions issued (fma chains, warp shuffles, loads, stores,
// conversions), the FP64 fma pipe, and a wave-quantisation efficiency.
#pragma once

#include <stdint.h>

namespace an5d {

struct Peaks {
    double hbm_gbs = 0;      // read + write bytes per second / 1e9
    double fp32_gflops = 0;  // 2 flops per fma
    double fp64_gflops = 0;
    double smem_gbs = 0;
    double sm_clock_mhz = 0;
    int sms = 0;
    int measured = 0;
};

struct ModelInput {
    int ndim, shape, radius, dtype, bt;
    int64_t nz, ny, nx;
    int tile_x, tile_y, tiles_x, tiles_y, hsn, stream_blocks, units, resident_units, sms;
};

// Peaks of the current device: measured ones if an5d_measure_peaks ran,
// otherwise nominal figures from the device attributes.
Peaks current_peaks();

// Predicted throughput in GCell-updates/s of a long run with this pass shape.
double model_gcells(const ModelInput &m);

}  // namespace an5d
