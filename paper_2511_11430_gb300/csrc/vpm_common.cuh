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

constexpr int P_F4 = 5;  // float4 per packed particle source
constexpr int S_F4 = 6;  // float4 per packed segment source

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
// Target boxes for the near/far test.  A warp's 64 targets (lane l holds index l
// in p0 and 32 + l in p1) are split at the largest jump between index-consecutive
// targets into two groups with one bounding box each, so that a warp straddling
// two distant runs of particles (say the end of one tip-vortex spiral and the
// start of the next) does not get one box spanning everything.  Boxes go to
// out[12] = {loA, hiA, loB, hiB} (xyz each); an empty group has lo = +inf.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_two_boxes(float3 p0, bool v0, float3 p1, bool v1, float* out)
{
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float3 n0, n1;
    n0.x = __shfl_down_sync(F, p0.x, 1), n0.y = __shfl_down_sync(F, p0.y, 1), n0.z = __shfl_down_sync(F, p0.z, 1);
    const float q0x = __shfl_sync(F, p1.x, 0), q0y = __shfl_sync(F, p1.y, 0), q0z = __shfl_sync(F, p1.z, 0);
    const bool nv0d = __shfl_down_sync(F, (int)v0, 1) != 0, q0v = __shfl_sync(F, (int)v1, 0) != 0;
    n1.x = __shfl_down_sync(F, p1.x, 1), n1.y = __shfl_down_sync(F, p1.y, 1), n1.z = __shfl_down_sync(F, p1.z, 1);
    const bool nv1d = __shfl_down_sync(F, (int)v1, 1) != 0;
    if (lane == 31) n0 = make_float3(q0x, q0y, q0z);
    const bool nv0 = lane == 31 ? q0v : nv0d;
    const bool nv1 = lane == 31 ? false : nv1d;
    float g0 = -1.f, g1 = -1.f;
    if (v0 && nv0) {
        const float dx = p0.x - n0.x, dy = p0.y - n0.y, dz = p0.z - n0.z;
        g0 = dx * dx + dy * dy + dz * dz;
    }
    if (v1 && nv1) {
        const float dx = p1.x - n1.x, dy = p1.y - n1.y, dz = p1.z - n1.z;
        g1 = dx * dx + dy * dy + dz * dz;
    }
    float g = g0;
    int k = lane;
    if (g1 > g) g = g1, k = 32 + lane;
    for (int o = 16; o > 0; o >>= 1) {
        const float og = __shfl_xor_sync(F, g, o);
        const int ok = __shfl_xor_sync(F, k, o);
        if (og > g || (og == g && ok < k)) g = og, k = ok;
    }
    // target index t goes to group A when t <= k (k = -1 would put all in B)
    const int ks = g >= 0.f ? k : -1;
    const float I = INFINITY;
    const bool a0 = v0 && lane <= ks, b0 = v0 && lane > ks;
    const bool a1 = v1 && 32 + lane <= ks, b1 = v1 && 32 + lane > ks;
    float lo[2][3], hi[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float x0 = c == 0 ? p0.x : (c == 1 ? p0.y : p0.z);
        const float x1 = c == 0 ? p1.x : (c == 1 ? p1.y : p1.z);
        lo[0][c] = fminf(a0 ? x0 : I, a1 ? x1 : I);
        hi[0][c] = fmaxf(a0 ? x0 : -I, a1 ? x1 : -I);
        lo[1][c] = fminf(b0 ? x0 : I, b1 ? x1 : I);
        hi[1][c] = fmaxf(b0 ? x0 : -I, b1 ? x1 : -I);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                lo[b][c] = fminf(lo[b][c], __shfl_xor_sync(F, lo[b][c], o));
                hi[b][c] = fmaxf(hi[b][c], __shfl_xor_sync(F, hi[b][c], o));
            }
    if (lane == 0)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 3; ++c) out[6 * b + c] = lo[b][c], out[6 * b + 3 + c] = hi[b][c];
    __syncwarp();
}

// Squared distance between box [lo, hi] and the tile box [tlo, thi] (0 when they overlap).
__device__ __forceinline__ float box_dist2(const float* lo, const float* hi, float4 tlo, float4 thi)
{
    const float dx = fmaxf(0.f, fmaxf(tlo.x - hi[0], lo[0] - thi.x));
    const float dy = fmaxf(0.f, fmaxf(tlo.y - hi[1], lo[1] - thi.y));
    const float dz = fmaxf(0.f, fmaxf(tlo.z - hi[2], lo[2] - thi.z));
    return dx * dx + dy * dy + dz * dz;
}

// Whether a tile box comes within sqrt(r2) of either of a warp's two boxes.
__device__ __forceinline__ bool boxes_near(const float* b12, float4 tlo, float4 thi, float r2)
{
    return box_dist2(b12, b12 + 3, tlo, thi) < r2 || box_dist2(b12 + 6, b12 + 9, tlo, thi) < r2;
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
