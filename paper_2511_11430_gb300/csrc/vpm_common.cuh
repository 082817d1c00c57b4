// Device-side helpers shared by the vortex-particle kernels (sm_103a).
//
// Packed FP32: Blackwell issues two FP32 operations per instruction on float2
// operands (FFMA2/FADD2/FMUL2).  Every pair kernel here holds two targets per
// thread in the .x and .y lanes of float2 registers, so one packed instruction
// advances two pair interactions; sources are broadcast from shared memory
// pre-duplicated into both lanes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vpm {

typedef float2 f2;

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    unsigned long long ua = *reinterpret_cast<unsigned long long*>(&a);
    unsigned long long ub = *reinterpret_cast<unsigned long long*>(&b);
    unsigned long long ud;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ud) : "l"(ua), "l"(ub));
    return *reinterpret_cast<f2*>(&ud);
}
__device__ __forceinline__ f2 splat(float v) { return make_float2(v, v); }
__device__ __forceinline__ f2 zero2() { return make_float2(0.f, 0.f); }

// Error-free transformation of a + b (Knuth's two-sum) on packed lanes:
// s = fl(a + b) and e such that s + e == a + b exactly.
__device__ __forceinline__ void two_sum2(f2 a, f2 b, f2& s, f2& e)
{
    s = add2(a, b);
    f2 bp = sub2(s, a);
    f2 ap = sub2(s, bp);
    e = add2(sub2(a, ap), sub2(b, bp));
}

// Compensated accumulator (hi, lo) += p.
__device__ __forceinline__ void fold2(f2& hi, f2& lo, f2 p)
{
    f2 s, e;
    two_sum2(hi, p, s, e);
    hi = s;
    lo = add2(lo, e);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// ---------------------------------------------------------------------------
// Device error word (one per device): bit flags latched by kernels.
// ---------------------------------------------------------------------------
enum : int { DEV_ERR_NONFINITE = 1, DEV_ERR_TIMEOUT = 2 };

// ---------------------------------------------------------------------------
// mbarrier + 1-D bulk async copy (global -> shared), the Blackwell/Hopper
// asynchronous copy engine path without a tensor map.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// One potentially blocking probe of a barrier phase: the hardware may suspend the
// thread for up to `hint_ns` until the phase completes, so waiting warps do not
// spin on the issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for a phase of `bar`: gives up (latching the device error word)
// once `limit_ns` of wall time has passed without the phase completing.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* dev_err, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity, 100000u)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity, 100000u)) return true;
        if (global_ns() - t0 > limit_ns) break;
    }
    atomicOr(dev_err, DEV_ERR_TIMEOUT);
    return false;
}

// ---------------------------------------------------------------------------
// Stream-K work split.  A sweep is a grid of (target tile t, source unit k)
// pairs; unit k < np is a particle tile of cost wp, else a segment tile of cost
// ws.  The cost line [0, TT*C) is cut into B equal ranges, block b owning the
// units whose start cost lies in [lo_b, hi_b).  A block therefore runs a
// contiguous run of units that may start and end inside target tiles; it writes
// one partial sum per target tile it touches, into slot b + t (unique because
// both b and the tiles it touches increase together).  The host keeps
// tot * B below 2^62 so that these products stay in 64-bit range.
// ---------------------------------------------------------------------------
struct StreamK {
    long long C;    // cost of one target tile
    long long tot;  // TT * C
    int TT, np, ns; // target tiles, particle units, segment units per target tile
    int wp, ws;     // unit costs
    int B;          // blocks

    __host__ __device__ long long lo(int b) const { return (long long)b * tot / B; }
    __host__ __device__ long long unit_start(int t, int k) const
    {
        return (long long)t * C + (k < np ? (long long)k * wp : (long long)np * wp + (long long)(k - np) * ws);
    }
    // First unit whose start cost is >= c (t == TT when none).
    __host__ __device__ void first_at_or_after(long long c, int& t, int& k) const
    {
        if (c >= tot) {
            t = TT;
            k = 0;
            return;
        }
        t = (int)(c / C);
        long long rem = c - (long long)t * C;
        long long pcost = (long long)np * wp;
        if (rem <= 0) {
            k = 0;
        } else if (rem <= pcost) {
            k = (int)((rem + wp - 1) / wp);  // may equal np: first segment unit
            if (k == np && ns == 0) {
                k = 0;
                ++t;
            }
        } else {
            long long r2 = rem - pcost;
            k = np + (int)((r2 + ws - 1) / ws);
            if (k >= np + ns) {
                k = 0;
                ++t;
            }
        }
    }
    // Block owning cost c.
    __host__ __device__ int block_of(long long c) const
    {
        return (int)(((c + 1) * (long long)B - 1) / tot);
    }
};

}  // namespace vpm
