// gtb_device.cuh -- device utilities shared by the gtb kernels (sm_103a).
//
//  * the device error word and bounded waits (no kernel ever spins forever or traps)
//  * mbarrier + TMA (cp.async.bulk.tensor) wrappers in inline PTX
//  * a binary64 reciprocal refined from the hardware approximation
//  * double-float ("df") arithmetic: an unevaluated sum hi + lo of two binary32
//    values carrying ~48 significant bits, on the FP32 pipe
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gtb {

// Set (never cleared by a kernel) when a bounded wait expires; read and
// cleared by gtb_device_status().
__device__ int g_device_error;

// Longest a thread waits on an mbarrier before giving up: 2 s of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Plain arrival (release semantics at CTA scope).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One try_wait on the phase with the given parity; true once it completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed, false (and the device error
// word set) when limit_ns (by default kWaitLimitNs) elapsed first.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > limit_ns) {
            atomicExch(&g_device_error, 1);
            return false;
        }
    }
    return true;
}

// The failure path of every bounded wait, exercised on purpose: one warp waits
// on an mbarrier that nobody arrives at (arrive = 0: the wait runs out after
// limit_ns, sets the device error word and the kernel returns normally) or that
// one thread completes first (arrive = 1: no error).
__global__ void selftest_wait_kernel(unsigned long long limit_ns, int arrive) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (arrive && threadIdx.x == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
    __syncwarp();
    mbar_wait(&bar, 0, limit_ns);
}

// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
// x (innermost) must be a multiple of 16 bytes / element size.
__device__ __forceinline__ void tma_load_3d(void *smem_dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (TMA) accesses of the same bytes.
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// f(idx, a, b) for the cells idx = tid, tid + NT, ... of a W x H region, a = idx % W,
// b = idx / W, the coordinates stepped by NT from cell to cell instead of divided anew.
template <int W, int H, int NT, typename F>
__device__ __forceinline__ void for_cells(int tid, F &&f) {
    constexpr int DA = NT % W, DB = NT / W;
    int a = tid % W, b = tid / W;
    for (int idx = tid; idx < W * H; idx += NT) {
        f(idx, a, b);
        a += DA, b += DB;
        if (a >= W) a -= W, ++b;
    }
}

// ---------------------------------------------------------------- async element copies
// One element global -> shared without a register round trip (cp.async): a block can
// have every copy of its staging in flight at once.  When !valid nothing is read and
// the destination is zero-filled (src-size 0); src must still be a valid address.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src, bool valid) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned n = valid ? (unsigned)sizeof(T) : 0u;
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_u32(dst)), "l"(src),
                 "n"((int)sizeof(T)), "r"(n)
                 : "memory");
}

// Wait for this thread's async element copies; they are then visible to this thread
// (other threads need a barrier as well).
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---------------------------------------------------------------- reciprocal
// a * b in binary64 (round to nearest) that stays inside its branch: volatile, so
// the compiler does not hoist it onto the FP64 pipe ahead of a rarely taken test.
__device__ __forceinline__ double mul_fp64(double a, double b) {
    double r;
    asm volatile("mul.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
    return r;
}

// 1/p in binary64: hardware seed (rcp.approx.ftz.f64) refined by one cubic
// Newton-Raphson step y <- y (1 + e + e^2), e = 1 - p y (the residual computed
// with one FMA, as in Markstein's division algorithms).  A seed accurate to
// 2^-k gives ~2^-3k before rounding, i.e. a result within ~1 ulp.
__device__ __forceinline__ double recip(double p) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(p));
    const double e = fma(-p, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

__device__ __forceinline__ float recip(float p) { return __frcp_rn(p); }

// ---------------------------------------------------------------- double-float
// Error-free transformations (Knuth, TAOCP vol. 2, 4.2.2: TwoSum; Dekker 1971:
// FastTwoSum; TwoProd via FMA) and the double-word algorithms of Joldes,
// Muller & Popescu, "Tight and rigorous error bounds for basic building blocks
// of double-word arithmetic", ACM TOMS 44(2), 2017.  All operations are
// written with explicit __f*_rn intrinsics so the compiler cannot contract or
// reassociate them.
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_from(float x) { return {x, 0.0f}; }

__device__ __forceinline__ float df_to_float(df a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// Double-word addition in the "sloppy" form (JMP17 Alg. 5): TwoSum of the high
// parts, the low parts added, one renormalisation.  Its absolute error is
// about 2u^2 (|x| + |y|) (u = 2^-24): like a binary64-style operation on the
// operands' magnitude, ample for the FP32-storage bound it serves (the
// column solve needs ~34 significant bits there), at 11 flops instead of 20.
__device__ __forceinline__ df operator+(df x, df y) {
    const df s = two_sum(x.hi, y.hi);
    const float v = __fadd_rn(x.lo, y.lo);
    const float w = __fadd_rn(s.lo, v);
    return fast_two_sum(s.hi, w);
}

__device__ __forceinline__ df operator-(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }

// double-word + word (JMP17 Alg. 4): relative error <= 2u^2.
__device__ __forceinline__ df operator+(df x, float y) {
    const df s = two_sum(x.hi, y);
    const float v = __fadd_rn(x.lo, s.lo);
    return fast_two_sum(s.hi, v);
}
__device__ __forceinline__ df operator-(df x, float y) { return x + (-y); }

// double-word x word (JMP17 Alg. 9): relative error <= 2u^2.
__device__ __forceinline__ df operator*(df x, float y) {
    const df c = two_prod(x.hi, y);
    const float cl3 = __fmaf_rn(x.lo, y, c.lo);
    return fast_two_sum(c.hi, cl3);
}

// double-word x double-word (JMP17 Alg. 12): relative error <= 5u^2.
__device__ __forceinline__ df operator*(df x, df y) {
    const df c = two_prod(x.hi, y.hi);
    float tl = __fmul_rn(x.hi, y.lo);
    tl = __fmaf_rn(x.lo, y.hi, tl);
    const float cl3 = __fadd_rn(c.lo, tl);
    return fast_two_sum(c.hi, cl3);
}

// Reciprocal of a double-word: th ~ 1/y.hi from the hardware approximation
// (rcp.approx.f32, within about one binary32 ulp), refined by one Newton step
// whose residual e = (1 - y.hi*th) - y.lo*th is formed with FMAs (the first
// product-difference is exact to within one rounding of a value of size
// ~2^-22); result th + th*e as a double-word, relative error ~2^-44.
__device__ __forceinline__ df recip(df y) {
    float th;
    asm("rcp.approx.f32 %0, %1;" : "=f"(th) : "f"(y.hi));
    float e = __fmaf_rn(-y.hi, th, 1.0f);
    e = __fmaf_rn(-y.lo, th, e);
    return fast_two_sum(th, __fmul_rn(th, e));
}

// Exact sum / difference of two binary32 values as a double-word (TwoSum).
__device__ __forceinline__ df df_add2(float a, float b) { return two_sum(a, b); }

// Fused double-word forms of x - y z and x + y z: the exact product of the high parts
// (TwoProd) with both cross terms added to its low part (y.lo z.lo, below u^2 |y z|,
// dropped), combined with x by a TwoSum of the high parts and the low parts' sum, then
// one renormalisation (FastTwoSum).  The product is not renormalised on its own, which
// saves four operations against the double-word product followed by the double-word
// sum (JMP17 Algs. 12 and 5), for an absolute error of the same order, a few
// u^2 (|x| + |y z|) with u = 2^-24.
__device__ __forceinline__ df df_fms(df x, df y, df z) {
    const float ph = __fmul_rn(y.hi, z.hi);
    float pl = __fmaf_rn(y.hi, z.hi, -ph);
    pl = __fmaf_rn(y.hi, z.lo, pl);
    pl = __fmaf_rn(y.lo, z.hi, pl);
    const df s = two_sum(x.hi, -ph);
    const float t = __fadd_rn(__fsub_rn(x.lo, pl), s.lo);
    return fast_two_sum(s.hi, t);
}
__device__ __forceinline__ df df_fma(df x, df y, df z) {
    return df_fms(x, -y, z);
}
// y z rounded once to binary32: the high product with both cross terms folded into
// one FMA chain (the error is within one binary32 rounding of the exact product).
__device__ __forceinline__ float df_mul_to_float(df y, df z) {
    return __fmaf_rn(y.hi, z.hi, __fmaf_rn(y.hi, z.lo, __fmul_rn(y.lo, z.hi)));
}

// ---------------------------------------------------------------- packed pairs
// Two binary32 values in one 64-bit register (the lower-addressed one in the low
// half, as a float2 in memory) and the paired instructions of the sm_100 family
// (add/sub/mul/fma .rn.f32x2): each half rounds exactly as the binary32 operation
// alone, so a thread runs two columns' arithmetic in one issue slot per operation
// with each column's result bit for bit that of the scalar form.
struct fpair {
    unsigned long long v;
};
__device__ __forceinline__ fpair fp_add(fpair a, fpair b) {
    fpair d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ fpair fp_sub(fpair a, fpair b) {
    fpair d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
// The product as fma(a, b, -0): the same value as the rounded product, sign included.
// The code generator fuses a paired multiply into a following paired add or subtract
// although both carry .rn (the scalar __fmul_rn never is), and it treats an fma whose
// addend is a literal -0 as a multiply; a __constant__ addend (which the host may
// rewrite, so neither compiler folds it) leaves nothing to fuse, and every operation
// keeps its own rounding, as in the scalar form.
__constant__ unsigned long long g_fp_negzero = 0x8000000080000000ull;
__device__ __forceinline__ fpair fp_mul(fpair a, fpair b) {
    fpair d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(g_fp_negzero));
    return d;
}
__device__ __forceinline__ fpair fp_fma(fpair a, fpair b, fpair c) {
    fpair d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
__device__ __forceinline__ fpair fp_neg(fpair a) { return fpair{a.v ^ 0x8000000080000000ull}; }
__device__ __forceinline__ fpair fp_make(float x, float y) {
    return fpair{(unsigned long long)__float_as_uint(x) | ((unsigned long long)__float_as_uint(y) << 32)};
}
__device__ __forceinline__ fpair fp_splat(float x) { return fp_make(x, x); }
__device__ __forceinline__ float fp_x(fpair a) { return __uint_as_float((unsigned)a.v); }
__device__ __forceinline__ float fp_y(fpair a) { return __uint_as_float((unsigned)(a.v >> 32)); }
__device__ __forceinline__ fpair fp_zero() { return fpair{0ull}; }

// Two columns' double-floats: the high parts in one pair, the low parts in the other;
// every operation is the df operation above, element by element.
struct dfpair {
    fpair hi, lo;
};
__device__ __forceinline__ dfpair two_sum(fpair a, fpair b) {
    const fpair s = fp_add(a, b);
    const fpair bb = fp_sub(s, a);
    const fpair e = fp_add(fp_sub(a, fp_sub(s, bb)), fp_sub(b, bb));
    return {s, e};
}
__device__ __forceinline__ dfpair fast_two_sum(fpair a, fpair b) {
    const fpair s = fp_add(a, b);
    return {s, fp_sub(b, fp_sub(s, a))};
}
__device__ __forceinline__ dfpair two_prod(fpair a, fpair b) {
    const fpair p = fp_mul(a, b);
    return {p, fp_fma(a, b, fp_neg(p))};
}
__device__ __forceinline__ dfpair operator+(dfpair x, dfpair y) {
    const dfpair s = two_sum(x.hi, y.hi);
    const fpair v = fp_add(x.lo, y.lo);
    const fpair w = fp_add(s.lo, v);
    return fast_two_sum(s.hi, w);
}
__device__ __forceinline__ dfpair operator-(dfpair x) { return {fp_neg(x.hi), fp_neg(x.lo)}; }
__device__ __forceinline__ dfpair operator-(dfpair x, dfpair y) { return x + (-y); }
__device__ __forceinline__ dfpair operator+(dfpair x, fpair y) {
    const dfpair s = two_sum(x.hi, y);
    const fpair v = fp_add(x.lo, s.lo);
    return fast_two_sum(s.hi, v);
}
__device__ __forceinline__ dfpair operator*(dfpair x, fpair y) {
    const dfpair c = two_prod(x.hi, y);
    const fpair cl3 = fp_fma(x.lo, y, c.lo);
    return fast_two_sum(c.hi, cl3);
}
__device__ __forceinline__ dfpair operator*(dfpair x, dfpair y) {
    const dfpair c = two_prod(x.hi, y.hi);
    fpair tl = fp_mul(x.hi, y.lo);
    tl = fp_fma(x.lo, y.hi, tl);
    const fpair cl3 = fp_add(c.lo, tl);
    return fast_two_sum(c.hi, cl3);
}
__device__ __forceinline__ dfpair recip(dfpair y) {
    float t0, t1;
    asm("rcp.approx.f32 %0, %1;" : "=f"(t0) : "f"(fp_x(y.hi)));
    asm("rcp.approx.f32 %0, %1;" : "=f"(t1) : "f"(fp_y(y.hi)));
    const fpair th = fp_make(t0, t1);
    fpair e = fp_fma(fp_neg(y.hi), th, fp_splat(1.0f));
    e = fp_fma(fp_neg(y.lo), th, e);
    return fast_two_sum(th, fp_mul(th, e));
}
__device__ __forceinline__ dfpair df_add2(fpair a, fpair b) { return two_sum(a, b); }
__device__ __forceinline__ dfpair df_fms(dfpair x, dfpair y, dfpair z) {
    const fpair ph = fp_mul(y.hi, z.hi);
    fpair pl = fp_fma(y.hi, z.hi, fp_neg(ph));
    pl = fp_fma(y.hi, z.lo, pl);
    pl = fp_fma(y.lo, z.hi, pl);
    const dfpair s = two_sum(x.hi, fp_neg(ph));
    const fpair t = fp_add(fp_sub(x.lo, pl), s.lo);
    return fast_two_sum(s.hi, t);
}
__device__ __forceinline__ dfpair df_fma(dfpair x, dfpair y, dfpair z) { return df_fms(x, -y, z); }
__device__ __forceinline__ fpair df_mul_to_float(dfpair y, dfpair z) {
    return fp_fma(y.hi, z.hi, fp_fma(y.hi, z.lo, fp_mul(y.lo, z.hi)));
}

// ---------------------------------------------------------------- streaming accesses
// Loads and stores with the streaming cache operator (ld/st.global.cs: lines allocated
// evict-first in L1 and L2) for data a kernel touches once: the column solve's inputs,
// its final outputs and the last read of its column state.  They leave L2 to the state
// that is written in the forward sweep and read back in the backward sweep.
template <typename T>
__device__ __forceinline__ T ld_once(const T *p) {
    return __ldcs(p);
}
template <>
__device__ __forceinline__ df ld_once<df>(const df *p) {
    const float2 v = __ldcs(reinterpret_cast<const float2 *>(p));
    return df{v.x, v.y};
}
template <>
__device__ __forceinline__ fpair ld_once<fpair>(const fpair *p) {
    return fpair{__ldcs(reinterpret_cast<const unsigned long long *>(p))};
}
// a pair of double-floats is stored as two consecutive df (the scalar layout)
template <>
__device__ __forceinline__ dfpair ld_once<dfpair>(const dfpair *p) {
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    return dfpair{fp_make(v.x, v.z), fp_make(v.y, v.w)};
}
template <typename T>
__device__ __forceinline__ void st_once(T *p, T v) {
    __stcs(p, v);
}
template <>
__device__ __forceinline__ void st_once<fpair>(fpair *p, fpair v) {
    __stcs(reinterpret_cast<unsigned long long *>(p), v.v);
}

// Drops the 128-byte L2 line at p (128-byte aligned, global memory) without writing
// it back (PTX discard.global.L2): its contents become undefined.  For column state
// whose last read has completed, so that the dead lines cost no DRAM write-back.
__device__ __forceinline__ void discard_l2_line(const void *p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(__cvta_generic_to_global(p)) : "memory");
}

}  // namespace gtb
