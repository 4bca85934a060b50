// paper_model.cu -- the paper's analytic performance model (Section 4), host only.
//
// The model classifies the threads of the paper's own kernel design (one
// thread per cell of a spatial block of bS_1 x ... x bS_{N-1} cells, one
// shared-memory write per thread and level, Table 3's shared-memory reads)
// and bounds a pass by the slowest of compute, global memory and shared
// memory, divided by an SM-utilisation efficiency.  It models the paper's
// V100/P100 kernels, not this library's GB300 kernels; the library ranks
// its own candidates with model.cu.  Readings of the text are noted where
// the model is stated in words only.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "an5d.h"
#include "an5d_internal.h"

namespace {

// Shared-memory reads per computing thread and level, Table 3 "Read
// (Practical)": star 2R (2D) / 4R (3D); box (2R+1)-1 (2D) / (2R+1)^2-1 (3D).
int smem_reads(int ndim, int shape, int R)
{
    if (shape == AN5D_STAR) return ndim == 2 ? 2 * R : 4 * R;
    const int p = 2 * R + 1;
    return ndim == 2 ? p - 1 : p * p - 1;
}

// Thread positions along one tiled axis, summed over its tiles (Section 3.1):
// tile k starts bT*R cells before its compute region R + k*c, c = bS - 2 bT R.
struct AxisCount {
    int64_t tiles = 0;
    int64_t oob = 0;                 // outside the padded grid
    int64_t boundary = 0;            // on the grid's halo (boundary conditions)
    int64_t interior = 0;            // inside the grid: redundant or valid
    int64_t valid = 0;               // inside the tile's compute region
    std::vector<int64_t> level;      // interior positions inside level t's valid region
};

AxisCount count_axis(int64_t I, int R, int bS, int bT)
{
    AxisCount a;
    const int c = bS - 2 * bT * R;
    a.tiles = (I + c - 1) / c;
    a.level.assign(bT + 1, 0);
    for (int64_t k = 0; k < a.tiles; ++k) {
        const int64_t s = R + k * c - (int64_t)bT * R;
        for (int j = 0; j < bS; ++j) {
            const int64_t x = s + j;
            if (x < 0 || x >= I + 2 * R) {
                ++a.oob;
            } else if (x < R || x >= I + R) {
                ++a.boundary;
            } else {
                ++a.interior;
                if (x >= s + (int64_t)bT * R && x < s + (int64_t)bT * R + c) ++a.valid;
                // the region of valid computation at level t: bS - 2 t R per axis
                for (int t = 1; t <= bT; ++t)
                    if (j >= t * R && j < bS - t * R) ++a.level[t];
            }
        }
    }
    return a;
}

}  // namespace

extern "C" int an5d_paper_model(const an5d_paper_stencil *st, const int64_t *dims, int bT,
                                const int *bS, int hSN, const an5d_paper_device *dev,
                                an5d_paper_model_result *out)
{
    using an5d::set_error;
    if (!st || !dims || !bS || !dev || !out) return set_error(AN5D_ERR_INVALID_ARG, "paper model: NULL argument");
    const int nd = st->ndim, R = st->radius;
    if ((nd != 2 && nd != 3) || R < 1 || R > 4 || (st->shape != AN5D_STAR && st->shape != AN5D_BOX) ||
        st->word_bytes <= 0 || bT < 1 || hSN < 1 || dev->sm_count < 1 || dev->max_threads_per_sm < 1 ||
        !(dev->peak_comp_gflops > 0) || !(dev->peak_gm_gbs > 0) || !(dev->peak_sm_gbs > 0))
        return set_error(AN5D_ERR_INVALID_ARG, "paper model: bad stencil, degree or device");
    const double ops = (double)st->op_fma + st->op_mul + st->op_add + st->op_other;
    if (ops <= 0 || st->op_fma < 0 || st->op_mul < 0 || st->op_add < 0 || st->op_other < 0)
        return set_error(AN5D_ERR_INVALID_ARG, "paper model: bad operation counts");
    for (int i = 0; i < nd; ++i)
        if (dims[i] < 1) return set_error(AN5D_ERR_INVALID_ARG, "paper model: dims must be >= 1");
    for (int i = 0; i < nd - 1; ++i)
        if (bS[i] - 2 * bT * R < 1)
            return set_error(AN5D_ERR_INVALID_ARG, "paper model: bS must exceed 2 bT R");

    // tiled axes: all but the streaming (slowest) one; bS[0] is the fastest (x)
    std::vector<AxisCount> ax;
    int64_t n_thr = 1;
    for (int i = 0; i < nd - 1; ++i) {
        ax.push_back(count_axis(dims[nd - 1 - i], R, bS[i], bT));
        n_thr *= bS[i];
    }
    double tot = 1, ingrid = 1, interior = 1, valid = 1;
    std::vector<double> lvl(bT + 1, 1.0);
    int64_t tiles = 1;
    for (const auto &a : ax) {
        tot *= (double)(a.oob + a.boundary + a.interior);
        ingrid *= (double)(a.boundary + a.interior);
        interior *= (double)a.interior;
        valid *= (double)a.valid;
        for (int t = 1; t <= bT; ++t) lvl[t] *= (double)a.level[t];
        tiles *= a.tiles;
    }
    const double boundary = ingrid - interior;

    // streaming axis: stream blocks of hSN output planes; level t of a block
    // covers its planes widened by (bT - t) R on each side (the redundant
    // planes of Section 3.2's division of the streaming dimension)
    const int64_t IN = dims[0];
    const int64_t nsb = (IN + hSN - 1) / hSN;
    double th_comp = 0, th_smr = 0, th_smw = 0, th_gmr = 0, th_gmw = 0;
    for (int64_t b = 0; b < nsb; ++b) {
        const int64_t z0 = R + b * hSN, z1 = std::min<int64_t>(z0 + hSN, IN + R);
        // T = 0: every in-grid thread loads one cell of each plane; every
        // thread (out-of-bound ones too) writes it to shared memory
        const int64_t l0 = std::max<int64_t>(0, z0 - (int64_t)bT * R);
        const int64_t l1 = std::min<int64_t>(IN + 2 * R, z1 + (int64_t)bT * R);
        const double np0 = (double)std::max<int64_t>(0, l1 - l0);
        th_gmr += np0 * ingrid;
        th_smw += np0 * tot;
        for (int t = 1; t <= bT; ++t) {
            const int64_t c0 = std::max<int64_t>(R, z0 - (int64_t)(bT - t) * R);
            const int64_t c1 = std::min<int64_t>(IN + R, z1 + (int64_t)(bT - t) * R);
            const double np = (double)std::max<int64_t>(0, c1 - c0);
            th_comp += np * lvl[t];                    // valid and redundant threads compute
            th_smr += np * (lvl[t] + boundary);        // boundary threads read shared memory too
            if (t < bT) th_smw += np * tot;            // the last level goes to global memory
        }
        th_gmw += (double)(z1 - z0) * valid;           // valid threads store level bT
    }

    const double w = st->word_bytes;
    const double flops = 2.0 * st->op_fma + st->op_mul + st->op_add + st->op_other;
    out->th_comp = th_comp;
    out->th_sm_read = th_smr;
    out->th_sm_write = th_smw;
    out->th_gm_read = th_gmr;
    out->th_gm_write = th_gmw;
    out->total_comp = th_comp * flops;
    out->total_gm = (th_gmr + th_gmw) * w;
    out->total_sm = (th_smr * smem_reads(nd, st->shape, R) + th_smw) * w;
    out->eff_alu = flops / (2.0 * ops);
    out->time_comp = out->total_comp / (dev->peak_comp_gflops * 1e9 * out->eff_alu);
    out->time_gm = out->total_gm / (dev->peak_gm_gbs * 1e9);
    out->time_sm = out->total_sm / (dev->peak_sm_gbs * 1e9);
    // SM utilisation: thread blocks resident per SM by the thread limit, and
    // the fraction of the last wave that is filled (reading of the formula)
    const int64_t per_sm = std::max<int64_t>(1, dev->max_threads_per_sm / n_thr);
    const double waves = (double)(tiles * nsb) / (double)(dev->sm_count * per_sm);
    out->eff_sm = waves / std::ceil(waves);
    out->n_tb = (int64_t)tiles * nsb;
    double tmax = out->time_comp;
    out->bound = 0;
    if (out->time_gm > tmax) tmax = out->time_gm, out->bound = 1;
    if (out->time_sm > tmax) tmax = out->time_sm, out->bound = 2;
    out->time_model = tmax / out->eff_sm;
    double cells = 1;
    for (int i = 0; i < nd; ++i) cells *= (double)dims[i];
    out->gcells = cells * bT / out->time_model / 1e9;
    out->gflops = out->gcells * flops;
    return set_error(AN5D_OK, "");
}
