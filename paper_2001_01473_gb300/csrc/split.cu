// split.cu -- halo-deepened domain split of one sweep into slabs.
//
// The overlapped tiling of Section 2.3 applied one level up: the grid is cut
// along its slowest axis into slabs, and each slab keeps bT*R ghost planes
// (the "halo of R*bT planes" a pass consumes) beyond the planes it owns on
// each side that borders another slab.  A pass of degree d <= bT then runs
// on every slab independently, as a plain sweep of the slab's own padded
// array whose outer R planes act as a fixed halo: the error that the stale
// outer planes introduce moves R planes per step, so after d steps it has
// reached (d-1)*R planes into the ghost region and none of the owned planes.
// One exchange per pass then refreshes every slab's ghost and outer planes
// from the slabs that own them.  The result is the single-grid result, bit
// for bit, because every owned cell sees the same chain of operations.
//
// This is the step a multi-GPU decomposition runs per device, with the
// exchange as peer copies between devices; here every slab lives on the
// calling device and the exchange is device-to-device copies on the caller's
// stream.  (No multi-device path is built: the library targets one GPU.)
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "an5d.h"
#include "an5d_internal.h"

namespace {

struct Slab {
    int64_t a, b;    // owned interior planes [a, b) (0-based interior index)
    int64_t lo, hi;  // padded planes [lo, hi) held by the slab's local array
};

// Slab k of nsub: an even split of the slow extent s (the first s % nsub
// slabs own one plane more), with `ghost` planes beyond each owned range
// and R halo planes outside them, clipped to the padded extent s + 2R.
Slab slab_of(int64_t s, int R, int64_t ghost, int nsub, int k)
{
    const int64_t q = s / nsub, r = s % nsub;
    Slab sl;
    sl.a = k * q + std::min<int64_t>(k, r);
    sl.b = sl.a + q + (k < r ? 1 : 0);
    sl.lo = std::max<int64_t>(0, sl.a + R - ghost - R);
    sl.hi = std::min<int64_t>(s + 2 * R, sl.b + R + ghost + R);
    return sl;
}

}  // namespace

using namespace an5d;

extern "C" int an5d_split_geometry(int ndim, const int64_t *dims, int radius, int bt, int nsub, int k,
                                   int64_t *out)
{
    if ((ndim != 2 && ndim != 3) || !dims || !out || radius < 1 || bt < 1 || nsub < 1 || k < 0 || k >= nsub)
        return set_error(AN5D_ERR_INVALID_ARG, "split geometry: ndim 2-3, radius and bT >= 1, 0 <= k < nsub");
    const int64_t s = dims[0];
    const int64_t ghost = (int64_t)bt * radius;
    if (s / nsub < ghost + radius)
        return set_error(AN5D_ERR_UNSUPPORTED,
                         "split: every slab must own at least bT*R + R planes of the slowest axis");
    const Slab sl = slab_of(s, radius, ghost, nsub, k);
    out[0] = sl.a;
    out[1] = sl.b;
    out[2] = sl.lo;
    out[3] = sl.hi;
    return AN5D_OK;
}

extern "C" int an5d_run_split(an5d_plan *plan, int nsub, const void *in, void *out, int64_t T, void *stream)
{
    PlanView v;
    if (int s = plan_view(plan, &v)) return s;
    if (!in || !out || T < 0 || nsub < 1) return set_error(AN5D_ERR_INVALID_ARG, "split: NULL buffer, T < 0 or nsub < 1");
    if (v.post != POST_NONE) return set_error(AN5D_ERR_UNSUPPORTED, "split: plain stencils only");
    if (((uintptr_t)in | (uintptr_t)out) & 15) return set_error(AN5D_ERR_INVALID_ARG, "split: buffers must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const int R = v.radius, bt = v.bt;
    const int64_t dims[3] = {v.ndim == 3 ? v.nz : v.ny, v.ndim == 3 ? v.ny : v.nx, v.nx};
    const int64_t s = dims[0];
    const size_t es = v.bytes / (size_t)v.total;
    const size_t plane = (size_t)(v.total / (s + 2 * R)) * es;  // bytes of one padded plane (2D: row)
    int64_t g[4];
    for (int k = 0; k < nsub; ++k)
        if (int st2 = an5d_split_geometry(v.ndim, dims, R, bt, nsub, k, g)) return st2;
    if (T == 0 || nsub == 1) return an5d_run(plan, in, out, T, stream);

    std::vector<Slab> sl(nsub);
    for (int k = 0; k < nsub; ++k) sl[k] = slab_of(s, R, (int64_t)bt * R, nsub, k);
    std::vector<an5d_plan *> lp(nsub, nullptr);
    std::vector<void *> buf(2 * (size_t)nsub, nullptr);
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (auto *p : lp) an5d_plan_destroy(p);
        for (void *b : buf) cudaFree(b);
    };
    int status = AN5D_OK;
    for (int k = 0; k < nsub && status == AN5D_OK; ++k) {
        int64_t ld[3] = {sl[k].hi - sl[k].lo - 2 * R, dims[1], dims[2]};
        lp[k] = an5d_plan_create(v.ndim, (an5d_shape)v.shape, R, v.coeffs, (an5d_dtype)v.dtype, ld);
        if (!lp[k]) {
            status = an5d_last_status();
            break;
        }
        if ((status = an5d_plan_set_config(lp[k], bt, v.hsn)) != AN5D_OK) break;
        const size_t bytes = (size_t)(sl[k].hi - sl[k].lo) * plane;
        for (int j = 0; j < 2 && status == AN5D_OK; ++j)
            if (cudaMalloc(&buf[2 * k + j], bytes) != cudaSuccess)
                status = set_error(AN5D_ERR_OOM, "split: slab buffers");
        // the slab's planes of the input, outer planes included
        if (status == AN5D_OK &&
            cudaMemcpyAsync(buf[2 * k], (const char *)in + sl[k].lo * plane, bytes, cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess)
            status = set_error(AN5D_ERR_CUDA, "split: slab copy");
    }
    // Pass list of Section 3.3: floor(T/bT) passes of bT, then one of T mod bT.
    std::vector<int> passes((size_t)(T / bt), bt);
    if (T % bt) passes.push_back((int)(T % bt));
    int cur = 0;  // buf[2k + cur] holds the slab's state at the start of a pass
    for (size_t pi = 0; pi < passes.size() && status == AN5D_OK; ++pi) {
        for (int k = 0; k < nsub && status == AN5D_OK; ++k)
            status = an5d_run(lp[k], buf[2 * k + cur], buf[2 * k + (cur ^ 1)], passes[pi], stream);
        if (status != AN5D_OK) break;
        cur ^= 1;
        // exchange: every plane a slab holds but does not own (its ghost and
        // outer planes, the global halo excepted) from the slab that owns it
        for (int k = 0; k < nsub && status == AN5D_OK; ++k) {
            const int64_t own0 = sl[k].a + R, own1 = sl[k].b + R;
            for (int j = 0; j < nsub && status == AN5D_OK; ++j) {
                if (j == k) continue;
                const int64_t src0 = sl[j].a + R, src1 = sl[j].b + R;  // planes slab j owns
                for (int side = 0; side < 2; ++side) {
                    const int64_t w0 = side == 0 ? sl[k].lo : own1, w1 = side == 0 ? own0 : sl[k].hi;
                    const int64_t c0 = std::max(w0, src0), c1 = std::min(w1, src1);
                    if (c1 <= c0) continue;
                    if (cudaMemcpyAsync((char *)buf[2 * k + cur] + (c0 - sl[k].lo) * plane,
                                        (const char *)buf[2 * j + cur] + (c0 - sl[j].lo) * plane,
                                        (size_t)(c1 - c0) * plane, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
                        status = set_error(AN5D_ERR_CUDA, "split: exchange copy");
                        break;
                    }
                }
            }
        }
    }
    // gather the owned planes; the global halo planes come from the input
    for (int k = 0; k < nsub && status == AN5D_OK; ++k) {
        const int64_t p0 = sl[k].a + R, p1 = sl[k].b + R;
        if (cudaMemcpyAsync((char *)out + p0 * plane, (const char *)buf[2 * k + cur] + (p0 - sl[k].lo) * plane,
                            (size_t)(p1 - p0) * plane, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            status = set_error(AN5D_ERR_CUDA, "split: gather");
    }
    if (status == AN5D_OK &&
        (cudaMemcpyAsync(out, in, (size_t)R * plane, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync((char *)out + (s + R) * plane, (const char *)in + (s + R) * plane, (size_t)R * plane,
                         cudaMemcpyDeviceToDevice, st) != cudaSuccess))
        status = set_error(AN5D_ERR_CUDA, "split: halo planes");
    int dev_status = AN5D_OK;
    if (status == AN5D_OK)
        for (int k = 0; k < nsub && dev_status == AN5D_OK; ++k) dev_status = an5d_plan_status(lp[k]);
    release();
    return status != AN5D_OK ? status : dev_status;
}
