// rism_internal.cuh -- internal types and device primitives of librism3d.
//
// Nothing here is part of the public ABI (include/rism3d.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "rism3d.h"

namespace rism {

constexpr int kMaxSites = RISM_MAX_SITES;

// Device error word written by kernels (first error wins).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_OVERFLOW = 2, DEV_BAD_INPUT = 3 };
struct DevErr {
    int code;
    int where;  // kernel id that reported it
};
enum : int { WHERE_DIRECT = 1, WHERE_TREE_EVAL = 2, WHERE_ADJOINT = 3, WHERE_BATCH = 4, WHERE_UPWARD = 5,
             WHERE_INPUT_CHECK = 6, WHERE_LRA = 7, WHERE_KSPACE = 8 };

// ---------------------------------------------------------------- records
// Atom geometry: position (physical A for the FP64 path; grid units relative
// to the grid origin for the FP32 path) and charge.
struct __align__(16) Geo {
    double x, y, z, q;
};
// Per (atom, site) Lennard-Jones terms, FP64 physical: A/d^12 - B/d^6 while d^2 < rc2.
struct __align__(16) LJd {
    double A, B, rc2, pad;
};
// Per (atom, site) Lennard-Jones terms, FP32 grid units: A/h^12, B/h^6, rc^2/h^2.
struct __align__(16) LJf {
    float A, B, rc2, pad;
};
// Source point for the FP32 kernels: position in grid units relative to the
// grid origin as float-float (hi + lo, |lo| <= ulp(hi)/2) and charge.  Grid
// point indices are exact small integers in FP32, so for a nearby source
// dx = (i - xh) - xl loses nothing in the first subtraction (Sterbenz) and
// carries one rounding of dx itself.  on_grid = 1 when the source sits
// exactly on a lattice point (only then can d = 0 occur).
struct __align__(16) SrcF {
    float xh, yh, zh, q;
    float xl, yl, zl, on_grid;
};

// Physical constants and per-site factors shared by every evaluation kernel.
struct Phys {
    int S;        // number of solvent sites
    double beta, k_e, eps_r, eta, kappa, a, ea2;
    double rs;    // short-range radius (A)
    double phi_c0, phi_h0;  // d -> 0 limits of erf(d/eta)/d and of the TCF kernel
    double qs[kMaxSites];
};

struct GridD {
    int nx, ny, nz;
    double h, ox, oy, oz;
};

// Raise, never lower, the dynamic shared-memory limit of a kernel on the current device.  The limit is a
// property of the function, not of a launch: lowering it for a small launch would leave a launch of the same
// kernel captured earlier in a graph (with more shared memory) over the limit whenever that node is launched
// on its own, as a profiler's replay does.
template <typename F>
cudaError_t raise_dyn_smem(F* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> cur;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& c = cur[{dev, reinterpret_cast<const void*>(kernel)}];
    if (bytes <= c) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) c = bytes;
    return e;
}

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two-wide FP32 arithmetic (sm_100 and later): one instruction applies the same IEEE round-to-nearest
// operation to both halves of a 64-bit register pair, so each half gets the result of the scalar op.
using f32x2 = unsigned long long;
__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 up2(f32x2 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// try_wait with a suspend-time hint: the waiting thread may sleep up to `ns` nanoseconds for the phase
// instead of returning at once, so a waiting warp issues few instructions.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return done != 0;
}
constexpr uint32_t kWaitSleepNs = 200;  // suspend hint per poll; limit polls x 200 ns bounds a wait
// Bounded wait: false when `limit` polls pass without the phase completing.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait_sleep(bar, parity, kWaitSleepNs)) return true;
    return false;
}
// One bulk (non-tensor) TMA copy global -> shared; dst, src 16-byte aligned,
// bytes a multiple of 16.  Completion is signalled on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void report_error(DevErr* e, int code, int where) {
    if (e && atomicCAS(&e->code, DEV_OK, code) == DEV_OK) e->where = where;
}

// Error-free transformation a + b = s + t (Knuth's TwoSum), used to fold FP32
// partial sums into a float-float accumulator.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float v) {
    float s = hi + v;
    float bb = s - hi;
    float t = (hi - (s - bb)) + (v - bb);
    hi = s;
    lo += t;
}

// float -> double on the integer pipe (the FP64 pipe of this part is slow).  Normal numbers: sign, exponent
// rebiased by 1023 - 127 = 896, fraction shifted left by 52 - 23 = 29.  The rare rest, out of line so that the
// common path stays short: all-ones exponent (infinity, NaN) kept all-ones, zero kept zero, a subnormal
// m 2^-149 renormalised from the position p of its leading bit as 2^(p - 149) (1 + f).
static __device__ __noinline__ double f2d_special(uint32_t b) {
    const uint32_t e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    unsigned long long r;
    if (e == 0xffu) {
        r = sign | (0x7ffull << 52) | ((unsigned long long)m << 29);
    } else if (m == 0u) {
        r = sign;
    } else {
        const int p = 31 - __clz((int)m);
        r = sign | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
    }
    return __longlong_as_double((long long)r);
}
__device__ __forceinline__ double f2d_alu(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if (__builtin_expect(e - 1u >= 254u, 0)) return f2d_special(b);
    const unsigned long long r = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)r);
}

// Error-free sum of two floats: a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Split a double into hi + lo floats (|lo| <= ulp(hi)/2).
__device__ __forceinline__ void split_ff(double v, float& hi, float& lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

__device__ __forceinline__ SrcF make_srcf(double x, double y, double z, double q) {
    SrcF s;
    split_ff(x, s.xh, s.xl);
    split_ff(y, s.yh, s.yl);
    split_ff(z, s.zh, s.zl);
    s.q = (float)q;
    s.on_grid = (x == floor(x) && y == floor(y) && z == floor(z)) ? 1.f : 0.f;
    return s;
}

}  // namespace rism
