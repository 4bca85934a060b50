// device_common.cuh -- sm_103a primitives shared by the sweep kernels:
// mbarrier + TMA (cp.async.bulk.tensor) row staging with bounded waits, and
// the per-point accumulation rules (plain fma chain, Dot2, binary16 rounding).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "an5d_internal.h"

namespace an5d {

constexpr unsigned FULL_MASK = 0xffffffffu;

// A bounded device wait gives up after this long, records AN5D_ERR_TIMEOUT in
// the plan's status word and lets the kernel return (no trap, no hang).
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Makes mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Raise the expected transaction bytes of the current phase without arriving.
__device__ __forceinline__ void mbar_expect_tx_only(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Warp-uniform bounded wait on an mbarrier phase.  Returns false (and sets
// the status word) when the limit is reached.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, int *status)
{
    if (__all_sync(FULL_MASK, mbar_try_wait(bar, parity))) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (__all_sync(FULL_MASK, mbar_try_wait(bar, parity))) return true;
        bool late = (global_ns() - t0) > WAIT_LIMIT_NS;
        if (__any_sync(FULL_MASK, late)) {
            if ((threadIdx.x & 31) == 0) atomicOr(status, STATUS_TIMEOUT);
            return false;
        }
    }
}

// One-dimensional tiled TMA load of `box` elements starting at element x of
// the tensor described by `map` into shared memory; completion is signalled
// on `bar` as transaction bytes.  x * sizeof(element) must be a multiple of
// 16 bytes; elements outside [0, extent) are filled with zeros.
__device__ __forceinline__ void tma_load_1d(void *dst, const CUtensorMap *map, int32_t x,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2}], [%3];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(smem_u32(bar))
        : "memory");
}

// Non-tensor bulk copy of `bytes` (a multiple of 16) from 16-byte aligned
// global memory to 16-byte aligned shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Acquire load of a global counter (pairs with a fenced atomic increment).
__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int pmod(int a, int m)
{
    int r = a % m;
    return r < 0 ? r + m : r;
}

// ----------------------------------------------------------------------------
// Storage / compute types.

template <typename S> struct StorageTraits;
template <> struct StorageTraits<float> {
    using C = float;
    static constexpr int ALIGN_ELEMS = 4;  // 16 bytes
};
template <> struct StorageTraits<double> {
    using C = double;
    static constexpr int ALIGN_ELEMS = 2;
};
template <> struct StorageTraits<__half> {
    using C = float;
    static constexpr int ALIGN_ELEMS = 8;
};

template <typename S>
__device__ __forceinline__ typename StorageTraits<S>::C load_c(S v)
{
    return v;
}
template <> __device__ __forceinline__ float load_c<__half>(__half v) { return __half2float(v); }

// V consecutive storage elements at p, converted to the compute type, read
// with the widest access the address's alignment allows.  A row staged by
// TMA keeps the global array's misalignment, so p's alignment is the same
// for every lane of a warp and the branch does not diverge; an aligned
// 16-byte read takes a quarter of the shared-memory wavefronts of four
// element reads at a 16-byte lane stride.  Generic form: element by element.
template <typename S, int V> struct CellLoader {
    static __device__ __forceinline__ void load(const S *p, typename StorageTraits<S>::C (&out)[V])
    {
#pragma unroll
        for (int v = 0; v < V; ++v) out[v] = load_c<S>(p[v]);
    }
};
template <> struct CellLoader<float, 4> {
    static __device__ __forceinline__ void load(const float *p, float (&out)[4])
    {
        const unsigned mis = (unsigned)reinterpret_cast<uintptr_t>(p) & 15u;
        if (mis == 0) {
            const float4 q = *reinterpret_cast<const float4 *>(p);
            out[0] = q.x, out[1] = q.y, out[2] = q.z, out[3] = q.w;
        } else if ((mis & 7u) == 0) {
            const float2 q0 = reinterpret_cast<const float2 *>(p)[0];
            const float2 q1 = reinterpret_cast<const float2 *>(p)[1];
            out[0] = q0.x, out[1] = q0.y, out[2] = q1.x, out[3] = q1.y;
        } else {
#pragma unroll
            for (int v = 0; v < 4; ++v) out[v] = p[v];
        }
    }
};
template <int V> struct CellLoader<double, V> {
    static __device__ __forceinline__ void load(const double *p, double (&out)[V])
    {
        if (V % 2 == 0 && ((unsigned)reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
#pragma unroll
            for (int i = 0; i < V / 2; ++i) {
                const double2 q = reinterpret_cast<const double2 *>(p)[i];
                out[2 * i] = q.x, out[2 * i + 1] = q.y;
            }
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = p[v];
        }
    }
};
template <typename S, int V>
__device__ __forceinline__ void load_cells(const S *p, typename StorageTraits<S>::C (&out)[V])
{
    CellLoader<S, V>::load(p, out);
}

template <typename S>
__device__ __forceinline__ S to_storage(typename StorageTraits<S>::C v)
{
    return v;
}
template <> __device__ __forceinline__ __half to_storage<__half>(float v)
{
    return __float2half_rn(v);
}

// Value kept for the next time level: binary16 storage rounds every level.
template <typename S>
__device__ __forceinline__ typename StorageTraits<S>::C level_round(typename StorageTraits<S>::C v)
{
    return v;
}
template <> __device__ __forceinline__ float level_round<__half>(float v)
{
    return __half2float(__float2half_rn(v));
}

// Correctly rounded primitives (never contracted or reassociated).
__device__ __forceinline__ float op_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double op_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float op_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double op_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float op_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double op_add(double a, double b) { return __dadd_rn(a, b); }
// IEEE division, round to nearest (CUDA's correctly rounded intrinsics).
__device__ __forceinline__ float op_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double op_div(double a, double b) { return __ddiv_rn(a, b); }

// Per-step operation of a division-type stencil on the finished weighted sum
// x: none, x / c (POST_DIV) or x * c with c the rounded reciprocal (POST_MUL).
template <int POST, typename C> __device__ __forceinline__ C post_op(C x, C c)
{
    if constexpr (POST == POST_DIV) return op_div(x, c);
    else if constexpr (POST == POST_MUL) return op_mul(x, c);
    else return x;
}
__device__ __forceinline__ float op_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double op_sub(double a, double b) { return __dsub_rn(a, b); }

enum : int { MODE_PLAIN = 0, MODE_DOT2 = 1 };

// Coefficients passed by value as a kernel parameter (constant bank).
template <typename C, int N> struct CoeffBlock {
    C c[N];
};

// Per-point accumulator.  PLAIN: acc = c0*f0, then acc = fma(ck, fk, acc).
// DOT2: Ogita-Rump-Oishi Dot2 -- TwoProduct by fma, TwoSum (Knuth), the
// error terms summed separately and added at the end.
template <int MODE, typename C> struct Acc;

template <typename C> struct Acc<MODE_PLAIN, C> {
    C v;
    __device__ __forceinline__ void first(C c, C f) { v = op_mul(c, f); }
    __device__ __forceinline__ void add(C c, C f) { v = op_fma(c, f, v); }
    __device__ __forceinline__ C result() const { return v; }
    __device__ __forceinline__ void set(C x) { v = x; }
};

template <typename C> struct Acc<MODE_DOT2, C> {
    C p, s;
    __device__ __forceinline__ void first(C c, C f)
    {
        p = op_mul(c, f);
        s = op_fma(c, f, -p);
    }
    __device__ __forceinline__ void add(C c, C f)
    {
        C h = op_mul(c, f);
        C r = op_fma(c, f, -h);
        C t = op_add(p, h);
        C z = op_sub(t, p);
        C q = op_add(op_sub(p, op_sub(t, z)), op_sub(h, z));
        p = t;
        s = op_add(s, op_add(q, r));
    }
    __device__ __forceinline__ C result() const { return op_add(p, s); }
    // A halo slot holds a fixed value: p = value, s = 0 gives it back exactly.
    __device__ __forceinline__ void set(C x)
    {
        p = x;
        s = C(0);
    }
};

// ----------------------------------------------------------------------------
// Packed pairs of binary32 (sm_100+ f32x2 arithmetic).  Each element of
// fma.rn.f32x2 / mul.rn.f32x2 is one IEEE operation rounded to nearest, so a
// packed chain gives the same bits as two scalar chains; it halves the issue
// slots the fma chain takes.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_pack(float lo, float hi)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// post_op on both halves of a packed pair; cp holds (c, c).
template <int POST> __device__ __forceinline__ f2_t f2_post(f2_t x, f2_t cp, float c)
{
    if constexpr (POST == POST_MUL) {
        return f2_mul(cp, x);
    } else if constexpr (POST == POST_DIV) {
        float lo, hi;
        f2_unpack(x, lo, hi);
        return f2_pack(op_div(lo, c), op_div(hi, c));
    } else {
        return x;
    }
}

// Store predicated by bit `bit` of `mask`, without a branch.
template <typename S> __device__ __forceinline__ void st_pred(S *p, S v, unsigned mask, int bit);
template <> __device__ __forceinline__ void st_pred<float>(float *p, float v, unsigned mask, int bit)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.f32 [%0], %1;\n\t}" ::"l"(p),
                 "f"(v), "r"(mask & (1u << bit))
                 : "memory");
}
template <> __device__ __forceinline__ void st_pred<double>(double *p, double v, unsigned mask, int bit)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.f64 [%0], %1;\n\t}" ::"l"(p),
                 "d"(v), "r"(mask & (1u << bit))
                 : "memory");
}
template <> __device__ __forceinline__ void st_pred<__half>(__half *p, __half v, unsigned mask, int bit)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.b16 [%0], %1;\n\t}" ::"l"(p),
                 "h"(__half_as_ushort(v)), "r"(mask & (1u << bit))
                 : "memory");
}

}  // namespace an5d
