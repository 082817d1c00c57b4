// Pair sweeps of the vortex-particle hot path on sm_103a.
//
//  * Gaussian-particle velocity and gradient (Eq. 2-4): u = sum_j K (Gamma_j x r),
//    J = [S x]/(4 pi) + sum_j H (Gamma_j x r) (x) r with S = sum_j K Gamma_j.
//  * Vatistas-cored straight segments (Sec. II.A), their velocity and exact gradient.
//  * Optionally the transposed stretching J^T Gamma_i of Eq. 5 per target.
//  * The stream-K reduction of per-warp partial sums and the per-target epilogue:
//    the velocity/gradient outputs, or the right-hand side of Eq. 4-5 (Vreman eddy
//    viscosity, stretching) formed in FP64 from the reduced sums.
//  * Particle strength exchange (the nu lap(Gamma) term of Eq. 5).
//
// Kernel organisation.  A thread owns two targets, kept in the two lanes of packed
// float2 registers so that each FFMA2/FADD2/FMUL2 advances two pair interactions.
// Sources are packed once per call into 128-source tiles (duplicated into both
// lanes, negated copies included so that every subtraction is an add).  The sweep
// block streams the tiles through a ring of shared-memory stages with the bulk-copy
// engine (cp.async.bulk completing on a per-stage "full" mbarrier); each of its 16
// warps waits on "full", reads every source by broadcast and counts itself out of
// the stage, and the last warp to leave a stage refills it with the tile six units
// ahead.  Warps drift freely within the ring and no block-wide barrier sits in the
// loop.  Work is split stream-K over
// (target tile, source tile) cost units so every SM gets the same cost however few
// targets there are.  Far from a warp's 64 targets (the tile's bounding box more
// than 7 sigma from both of the warp's two target boxes) the blob kernel equals
// the point-vortex kernel to FP32 precision, so far tiles run the 1/r^3 form with
// one rsqrt; near tiles evaluate the regularised kernel exactly per pair.  Each tile's sums start from zero and are folded into a
// per-thread running sum kept in shared memory: a compensated (hi, lo) pair with
// Knuth's two-sum, or a plain sum, so long source lists keep a tile-sized error.
#include <math.h>

#include <mutex>

#include "vpm_common.cuh"
#include "vpm_internal.h"
#include "vpm_kernel.cuh"

namespace vpm {

// The sources of a particle tile.  The velocity-only loop is unrolled twice; the
// gradient loop, whose body already holds enough independent work, is not (measured:
// unrolling it costs 3.5%, unrolling the velocity loop gains 7%).
template <bool GRAD, bool STRETCH, bool NEAR>
__device__ __forceinline__ void particle_tile(Acc<GRAD, STRETCH>& a, const float4* __restrict__ s, int cnt, f2 X,
                                              f2 Y, f2 Z, const NearConst& nc, const Own& o)
{
    if constexpr (GRAD) {
#pragma unroll 1
        for (int j = 0; j < cnt; ++j) particle_source<GRAD, STRETCH, NEAR>(a, s + j * P_F4, X, Y, Z, nc, o);
    } else {
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) particle_source<GRAD, STRETCH, NEAR>(a, s + j * P_F4, X, Y, Z, nc, o);
    }
}

// The tile's sums without stretching (a far particle tile or a segment tile) into the
// fold rows of the stretching sweep: rows 0..13 copied, rows 14..16 set to the tile's
// transposed stretching J_tile^T Gamma_i (times 4 pi), formed from its partial S and
// G' -- for these tiles the two terms do not cancel.  The target's own strength is
// read here, after the tile's loop, so that it is not held in registers through it.
template <bool GRAD, bool STRETCH>
__device__ __forceinline__ void finish_tile(Acc<GRAD, STRETCH>& a, const Acc<GRAD, false>& t, const float4* tstr,
                                            int i0, int i1, int n_tgt)
{
    static_assert(GRAD || !STRETCH, "stretching needs the gradient sums");
#pragma unroll
    for (int q = 0; q < Acc<GRAD, false>::N; ++q) a.v[q] = t.v[q];
    if constexpr (STRETCH) {
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
    if (i0 < n_tgt) g0 = tstr[i0];
    if (i1 < n_tgt) g1 = tstr[i1];
    const f2 ogx = make_float2(g0.x, g1.x), ogy = make_float2(g0.y, g1.y), ogz = make_float2(g0.z, g1.z);
    const f2 Sx = t.v[3], Sy = t.v[4], Sz = t.v[5];
    const f2 Gxx = t.v[6], Gxy = t.v[7], Gxz = t.v[8], Gyx = t.v[9], Gyy = t.v[10], Gyz = t.v[11], Gzx = t.v[12],
             Gzy = t.v[13];
    const f2 Gzz = mul2(add2(Gxx, Gyy), splat(-1.f));
    const f2 m3 = splat(-3.f);
    // Gamma_i x S - 3 G'^T Gamma_i
    const f2 tx = sub2(mul2(ogy, Sz), mul2(ogz, Sy));
    const f2 ty = sub2(mul2(ogz, Sx), mul2(ogx, Sz));
    const f2 tz = sub2(mul2(ogx, Sy), mul2(ogy, Sx));
    const f2 gx = fma2(Gzx, ogz, fma2(Gyx, ogy, mul2(Gxx, ogx)));
    const f2 gy = fma2(Gzy, ogz, fma2(Gyy, ogy, mul2(Gxy, ogx)));
    const f2 gz = fma2(Gzz, ogz, fma2(Gyz, ogy, mul2(Gxz, ogx)));
    a.v[14] = fma2(m3, gx, tx);
    a.v[15] = fma2(m3, gy, ty);
    a.v[16] = fma2(m3, gz, tz);
    }
}

// ---------------------------------------------------------------------------
// Packing kernels (one thread per source slot, 128 per block = one tile).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SRC_TILE) pack_particles_kernel(const float4* __restrict__ pos,
                                                                  const float4* __restrict__ str, int n,
                                                                  float4* __restrict__ out, float4* __restrict__ box)
{
    const int j = blockIdx.x * SRC_TILE + threadIdx.x;
    const bool valid = j < n;
    float x = 0.f, y = 0.f, z = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    if (valid) {
        const float4 p = pos[j], g = str[j];
        x = p.x, y = p.y, z = p.z;
        gx = g.x, gy = g.y, gz = g.z;
    }
    float4* o = out + (size_t)j * P_F4;
    o[0] = make_float4(-x, -x, -y, -y);
    o[1] = make_float4(-z, -z, gx, gx);
    o[2] = make_float4(gy, gy, gz, gz);
    o[3] = make_float4(-gx, -gx, -gy, -gy);
    o[4] = make_float4(-gz, -gz, 0.f, 0.f);
    float lo[3] = {valid ? x : INFINITY, valid ? y : INFINITY, valid ? z : INFINITY};
    float hi[3] = {valid ? x : -INFINITY, valid ? y : -INFINITY, valid ? z : -INFINITY};
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o2));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o2));
        }
    __shared__ float sb[SRC_TILE / 32][6];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 3; ++c) sb[w][c] = lo[c], sb[w][3 + c] = hi[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int ww = 1; ww < SRC_TILE / 32; ++ww)
            for (int c = 0; c < 3; ++c) lo[c] = fminf(lo[c], sb[ww][c]), hi[c] = fmaxf(hi[c], sb[ww][3 + c]);
        box[2 * blockIdx.x] = make_float4(lo[0], lo[1], lo[2], 0.f);
        box[2 * blockIdx.x + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
}

__global__ void __launch_bounds__(SRC_TILE) pack_segments_kernel(const float4* __restrict__ sa,
                                                                 const float4* __restrict__ sb, int m, float core,
                                                                 int vn, int rings, float4* __restrict__ out,
                                                                 float4* __restrict__ box)
{
    const int j = blockIdx.x * SRC_TILE + threadIdx.x;
    const bool valid = j < m;
    float ax = 0.f, ay = 0.f, az = 0.f, rx = 1.f, ry = 0.f, rz = 0.f, g = 0.f;
    float4 bb = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        const float4 a = sa[j];
        bb = sb[j];
        ax = a.x, ay = a.y, az = a.z;
        rx = bb.x - a.x, ry = bb.y - a.y, rz = bb.z - a.z;
        g = a.w;
    }
    const float L2 = rx * rx + ry * ry + rz * rz;
    const float cl2 = core * core * L2;
    float e = vn == 2 ? cl2 * cl2 : cl2;
    if (!(L2 > 0.f)) g = 0.f, e = 1.f;  // a zero-length segment induces nothing; keeps D > 0
    // Closed four-sided rings: in every group of four segments of the tile, each one's
    // end point is the next one's start point (k -> k + 1 mod 4), bit for bit; groups
    // wholly past the end do not count.  Such a tile is packed by ring.
    const int lane = threadIdx.x & 31, nxt = (lane & ~3) | ((lane + 1) & 3);
    const float nax = __shfl_sync(0xffffffffu, ax, nxt), nay = __shfl_sync(0xffffffffu, ay, nxt),
                naz = __shfl_sync(0xffffffffu, az, nxt);
    const bool joins = valid && __float_as_uint(bb.x) == __float_as_uint(nax) &&
                       __float_as_uint(bb.y) == __float_as_uint(nay) && __float_as_uint(bb.z) == __float_as_uint(naz);
    const unsigned vmask = __ballot_sync(0xffffffffu, valid), jmask = __ballot_sync(0xffffffffu, joins);
    const int g4 = lane & ~3;
    const bool ring_ok = ((vmask >> g4) & 0xFu) == 0u || ((jmask >> g4) & 0xFu) == 0xFu;
    const bool closed = __syncthreads_and(ring_ok && rings) != 0;
    if (closed) {
        float2* o2 = reinterpret_cast<float2*>(out + (size_t)blockIdx.x * SRC_TILE * S_F4) + (threadIdx.x >> 2) * 48;
        const int k = threadIdx.x & 3;
        o2[3 * k] = make_float2(-ax, -ax);
        o2[3 * k + 1] = make_float2(-ay, -ay);
        o2[3 * k + 2] = make_float2(-az, -az);
        o2[12 + 3 * k] = make_float2(rx, rx);
        o2[13 + 3 * k] = make_float2(ry, ry);
        o2[14 + 3 * k] = make_float2(rz, rz);
        o2[24 + 3 * k] = make_float2(-rx, -rx);
        o2[25 + 3 * k] = make_float2(-ry, -ry);
        o2[26 + 3 * k] = make_float2(-rz, -rz);
        o2[36 + 2 * k] = make_float2(L2, L2);
        o2[37 + 2 * k] = make_float2(e, e);
        o2[44 + k] = make_float2(g, g);
    } else {
        float4* o = out + (size_t)j * S_F4;
        o[0] = make_float4(-ax, -ax, -ay, -ay);
        o[1] = make_float4(-az, -az, rx, rx);
        o[2] = make_float4(ry, ry, rz, rz);
        o[3] = make_float4(-rx, -rx, -ry, -ry);
        o[4] = make_float4(-rz, -rz, -L2, -L2);
        o[5] = make_float4(g, g, e, e);
    }
    // tile box of both end points, and the longest segment (in lo.w)
    const float bx = ax + rx, by = ay + ry, bz = az + rz;
    float lo[4] = {valid ? fminf(ax, bx) : INFINITY, valid ? fminf(ay, by) : INFINITY,
                   valid ? fminf(az, bz) : INFINITY, valid ? -sqrtf(L2) : 0.f};
    float hi[3] = {valid ? fmaxf(ax, bx) : -INFINITY, valid ? fmaxf(ay, by) : -INFINITY,
                   valid ? fmaxf(az, bz) : -INFINITY};
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o2));
#pragma unroll
        for (int c = 0; c < 3; ++c) hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o2));
    }
    __shared__ float sbx[SRC_TILE / 32][7];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        for (int c = 0; c < 4; ++c) sbx[w][c] = lo[c];
        for (int c = 0; c < 3; ++c) sbx[w][4 + c] = hi[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int ww = 1; ww < SRC_TILE / 32; ++ww) {
            for (int c = 0; c < 4; ++c) lo[c] = fminf(lo[c], sbx[ww][c]);
            for (int c = 0; c < 3; ++c) hi[c] = fmaxf(hi[c], sbx[ww][4 + c]);
        }
        box[2 * blockIdx.x] = make_float4(lo[0], lo[1], lo[2], -lo[3]);
        box[2 * blockIdx.x + 1] = make_float4(hi[0], hi[1], hi[2], closed ? 1.f : 0.f);
    }
}

// ---------------------------------------------------------------------------
// The stream-K sweep: SWEEP_CW warps per block sharing a ring of source stages.
// ---------------------------------------------------------------------------
struct SweepArgs {
    const float4* tgt;
    const float4* tstr;  // target strengths (stretching), may be null
    int n_tgt;
    const float4* psrc;
    const float4* pbox;
    int n_src;
    const float4* ssrc;
    const float4* sbox;
    int m_seg;
    int vn;
    int core_pos;  // the segment core is > 0
    StreamK sk;
    NearConst nc;
    float* part;
    int* dev_err;
};

constexpr int BUF_F4 = SRC_TILE * S_F4 + 2;  // the larger tile format + the tile's bounding box
constexpr uint64_t WAIT_LIMIT = 2000000000ull;  // 2 s of wall time

template <bool GRAD, bool STRETCH>
__host__ __device__ constexpr int n_rows()
{
    return Acc<GRAD, STRETCH>::N;
}

// Dynamic shared memory: SWEEP_STAGES source tiles, then the running sums of the
// consumer threads, [row][hi|lo][thread] as float2 (the two targets).
template <bool GRAD, bool COMP, bool STRETCH>
__host__ __device__ constexpr size_t sweep_smem_bytes()
{
    return (size_t)SWEEP_STAGES * BUF_F4 * 16 + (size_t)n_rows<GRAD, STRETCH>() * (COMP ? 2 : 1) * SWEEP_CW * 32 * 8;
}

// KIND: the source tiles a launch sweeps.  SWEEP_PARTICLES takes particle tiles and,
// in the one-launch plan of small problems, segment tiles one segment at a time;
// SWEEP_SEGMENTS takes only segment tiles, including those packed as closed rings.
// The ring loop needs more registers than the particle loop; in a launch of its own
// it costs the particle tiles nothing.  (Measured: the particle launch compiled
// without its segment loop is allocated fewer registers and runs 4% slower.)
constexpr int SWEEP_PARTICLES = 0, SWEEP_SEGMENTS = 1;

template <bool GRAD, bool COMP, bool STRETCH, int KIND>
__global__ void __launch_bounds__(SWEEP_TPB, 1) sweep_kernel(const SweepArgs A)
{
    extern __shared__ __align__(128) float4 dsm[];
    __shared__ __align__(8) uint64_t full[SWEEP_STAGES];
    __shared__ int released[SWEEP_STAGES];
    __shared__ int issued_round[SWEEP_STAGES];  // round of the latest copy into each stage
    __shared__ float wbox[SWEEP_CW][12];
    constexpr int NR = n_rows<GRAD, STRETCH>();
    constexpr int NT = SWEEP_CW * 32;
    float4* stage = dsm;
    f2* run = reinterpret_cast<f2*>(dsm + SWEEP_STAGES * BUF_F4);  // [NR][COMP?2:1][NT]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const StreamK& sk = A.sk;
    const int b = blockIdx.x;
    const long long lo_b = sk.lo(b), hi_b = sk.lo(b + 1);
    int t0, k0;
    sk.first_at_or_after(lo_b, t0, k0);
    if (t0 >= sk.TT || sk.unit_start(t0, k0) >= hi_b) return;  // block owns no unit (uniform)
    const int nunits = sk.np + sk.ns;

    // Copies source unit kk (and its bounding box) into stage s, completing on full[s].
    auto issue = [&](int kk, int s, int round) {
        issued_round[s] = round;
        fence_proxy_async_smem();
        if (kk < sk.np) {
            const uint32_t bytes = SRC_TILE * P_F4 * 16;
            mbar_expect_tx(&full[s], bytes + 32);
            bulk_g2s(stage + (size_t)s * BUF_F4, A.psrc + (size_t)kk * SRC_TILE * P_F4, bytes, &full[s]);
            bulk_g2s(stage + (size_t)s * BUF_F4 + SRC_TILE * S_F4, A.pbox + 2 * kk, 32, &full[s]);
        } else {
            const uint32_t bytes = SRC_TILE * S_F4 * 16;
            mbar_expect_tx(&full[s], bytes + 32);
            bulk_g2s(stage + (size_t)s * BUF_F4, A.ssrc + (size_t)(kk - sk.np) * SRC_TILE * S_F4, bytes, &full[s]);
            bulk_g2s(stage + (size_t)s * BUF_F4 + SRC_TILE * S_F4, A.sbox + 2 * (kk - sk.np), 32, &full[s]);
        }
    };
    // The unit `ahead` places after (t, k) in this block's run, if the block owns it.
    auto unit_ahead = [&](int t, int k, int ahead, int& kk) {
        for (int q = 0; q < ahead; ++q)
            if (++k == nunits) k = 0, ++t;
        kk = k;
        return t < sk.TT && sk.unit_start(t, k) < hi_b;
    };

    if (tid == 0) {
        for (int s = 0; s < SWEEP_STAGES; ++s) {
            mbar_init(&full[s], 1);
            released[s] = 0;
        }
        mbar_fence_init();
        for (int s = 0; s < SWEEP_STAGES; ++s) {  // first fill of the ring
            int kk;
            if (!unit_ahead(t0, k0, s, kk)) break;
            issue(kk, s, 0);
        }
    }
    __syncthreads();

    // ---------------- consumers ----------------
    const int ct = warp * 32 + lane;  // consumer thread index
    Acc<GRAD, STRETCH> acc;
    f2 X = zero2(), Y = zero2(), Z = zero2();
    int t = t0, k = k0, cur_t = -1;
    auto zero_run = [&]() {
#pragma unroll
        for (int q = 0; q < NR * (COMP ? 2 : 1); ++q) run[q * NT + ct] = zero2();
    };
    zero_run();
    for (int i = 0;; ++i) {
        const int s = i % SWEEP_STAGES, r = i / SWEEP_STAGES;
        int nt = t, nk = k + 1;
        if (nk == nunits) {
            nk = 0;
            ++nt;
        }
        const bool has_next = nt < sk.TT && sk.unit_start(nt, nk) < hi_b;
        if (t != cur_t) {  // new target tile: this warp's 64 targets, their box and strengths
            cur_t = t;
            const int i0 = t * TGT_TILE + warp * 64 + lane, i1 = i0 + 32;
            float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0;
            const bool v0 = i0 < A.n_tgt, v1 = i1 < A.n_tgt;
            if (v0) p0 = A.tgt[i0];
            if (v1) p1 = A.tgt[i1];
            X = make_float2(p0.x, p1.x);
            Y = make_float2(p0.y, p1.y);
            Z = make_float2(p0.z, p1.z);
            warp_two_boxes(make_float3(p0.x, p0.y, p0.z), v0, make_float3(p1.x, p1.y, p1.z), v1, wbox[warp]);
        }
        if (!mbar_wait_bounded(&full[s], r & 1, A.dev_err, WAIT_LIMIT)) {
            // latched; the results are invalid.  Let this block's copies in flight land
            // (bounded) before its shared memory is released, then leave.
            if (lane == 0)
                for (int q = 0; q < SWEEP_STAGES; ++q)
                    mbar_wait_bounded(&full[q], issued_round[q] & 1, A.dev_err, WAIT_LIMIT);
            break;
        }

        const float4* src = stage + (size_t)s * BUF_F4;
        // Far particle tiles and segment tiles accumulate without the stretching rows and
        // the target strengths (fewer live registers in their loops); finish_tile adds the
        // stretching from the tile's sums afterwards.  Near particle tiles accumulate the
        // stretching pair by pair (it cancels there) with the strengths loaded for them.
        const int ti0 = t * TGT_TILE + warp * 64 + lane, ti1 = ti0 + 32;
        if (KIND == SWEEP_PARTICLES && k < sk.np) {
            const int cnt = min(SRC_TILE, A.n_src - k * SRC_TILE);
            const float4 tlo = src[SRC_TILE * S_F4], thi = src[SRC_TILE * S_F4 + 1];
            if (boxes_near(wbox[warp], tlo, thi, A.nc.far2)) {
                Own own{zero2(), zero2(), zero2()};
                if (STRETCH) {
                    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
                    if (ti0 < A.n_tgt) g0 = A.tstr[ti0];
                    if (ti1 < A.n_tgt) g1 = A.tstr[ti1];
                    own.gx = make_float2(g0.x, g1.x);
                    own.gy = make_float2(g0.y, g1.y);
                    own.gz = make_float2(g0.z, g1.z);
                }
                acc.zero();
                particle_tile<GRAD, STRETCH, true>(acc, src, cnt, X, Y, Z, A.nc, own);
            } else {
                Acc<GRAD, false> tf;
                tf.zero();
                particle_tile<GRAD, false, false>(tf, src, cnt, X, Y, Z, A.nc, Own{});
                finish_tile<GRAD, STRETCH>(acc, tf, A.tstr, ti0, ti1, A.n_tgt);
            }
        } else {
            const int cnt = min(SRC_TILE, A.m_seg - (k - sk.np) * SRC_TILE);
            const float4 tlo = src[SRC_TILE * S_F4], thi = src[SRC_TILE * S_F4 + 1];
            const float margin = 1e-3f * tlo.w;
            const bool safe = A.core_pos && margin > 0.f && !boxes_near(wbox[warp], tlo, thi, margin * margin);
            Acc<GRAD, false> tf;
            tf.zero();
            if (KIND == SWEEP_SEGMENTS && thi.w != 0.f) {  // closed four-sided rings, packed by corner
                if (safe)
                    ring_tile<GRAD, true>(tf, src, cnt >> 2, X, Y, Z, A.vn);
                else
                    ring_tile<GRAD, false>(tf, src, cnt >> 2, X, Y, Z, A.vn);
            } else if (safe) {
                segment_tile<GRAD, false, true>(tf, src, cnt, X, Y, Z, A.vn);
            } else {
                segment_tile<GRAD, false, false>(tf, src, cnt, X, Y, Z, A.vn);
            }
            finish_tile<GRAD, STRETCH>(acc, tf, A.tstr, ti0, ti1, A.n_tgt);
        }
        __syncwarp();
        if (lane == 0) {  // the last warp to finish with stage s refills it with unit i + SWEEP_STAGES
            __threadfence_block();
            if (atomicAdd(&released[s], 1) == SWEEP_CW - 1) {
                released[s] = 0;
                __threadfence_block();
                int kk;
                if (unit_ahead(t, k, SWEEP_STAGES, kk)) issue(kk, s, r + 1);
            }
        }
        // fold this tile's sums into the running sums
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            if (COMP) {
                f2 hi = run[(2 * q) * NT + ct], lo = run[(2 * q + 1) * NT + ct];
                fold2(hi, lo, acc.v[q]);
                run[(2 * q) * NT + ct] = hi;
                run[(2 * q + 1) * NT + ct] = lo;
            } else {
                run[q * NT + ct] = add2(run[q * NT + ct], acc.v[q]);
            }
        }
        if (!has_next || nt != t) {  // this warp's partial of target tile t
            float* P = A.part + ((size_t)(b + t) * (COMP ? 2 * NR : NR)) * TGT_TILE + warp * 64 + lane;
#pragma unroll
            for (int q = 0; q < NR * (COMP ? 2 : 1); ++q) {
                const f2 v = run[q * NT + ct];
                // rows: hi of every accumulator first, then lo
                const int row = COMP ? ((q & 1) ? NR + (q >> 1) : (q >> 1)) : q;
                P[(size_t)row * TGT_TILE] = v.x;
                P[(size_t)row * TGT_TILE + 32] = v.y;
            }
            zero_run();
        }
        if (!has_next) break;
        t = nt;
        k = nk;
    }
}

// ---------------------------------------------------------------------------
// Reduction of the stream-K partial sums (fixed order, FP64) and epilogue.
// ---------------------------------------------------------------------------
struct EpiArgs {
    StreamK sk, sks;  // the particle and the segment launch
    const float* part;
    const float* part_s;
    int n, ncomp, comp;
    EpilogueOut o;
    int* dev_err;
};

__device__ __forceinline__ void check_finite(int* dev_err, double v)
{
    if (!isfinite(v)) atomicOr(dev_err, DEV_ERR_NONFINITE);
}

__global__ void __launch_bounds__(256) epilogue_kernel(const EpiArgs E)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= E.n) return;
    const int t = i / TGT_TILE, l = i % TGT_TILE;
    // The partial sums are folded in FP32 double-float arithmetic (hi by Knuth's
    // two-sum, the low words added apart: about 48 bits) and converted to FP64 once
    // per row; the FP64 pipe, a small fraction of the FP32 rate here, keeps only the
    // per-target algebra below.
    float H[17], Lw[17];
#pragma unroll
    for (int c = 0; c < 17; ++c) H[c] = 0.f, Lw[c] = 0.f;
    // the partial sums of the particle launch, then those of the segment launch
    for (int launch = 0; launch < 2; ++launch) {
        const StreamK& sk = launch ? E.sks : E.sk;
        const float* part = launch ? E.part_s : E.part;
        const int nunits = sk.np + sk.ns;
        if (nunits == 0) continue;
        const int b0 = sk.block_of(sk.unit_start(t, 0));
        const int b1 = sk.block_of(sk.unit_start(t, nunits - 1));
        const int rows = E.comp ? 2 * E.ncomp : E.ncomp;
        for (int b = b0; b <= b1; ++b) {
            const long long lo_b = sk.lo(b), hi_b = sk.lo(b + 1);
            long long c0 = lo_b > (long long)t * sk.C ? lo_b : (long long)t * sk.C;
            int tt, kk;
            sk.first_at_or_after(c0, tt, kk);
            if (tt != t || sk.unit_start(tt, kk) >= hi_b) continue;  // block b ran no unit of tile t
            const float* P = part + (size_t)(b + t) * rows * TGT_TILE + l;
#pragma unroll
            for (int c = 0; c < 17; ++c) {  // a constant bound keeps the sums in registers
                if (c < E.ncomp) {
                    float sum, err;
                    two_sum(H[c], P[(size_t)c * TGT_TILE], sum, err);
                    H[c] = sum;
                    Lw[c] = __fadd_rn(Lw[c], err);
                    if (E.comp) Lw[c] = __fadd_rn(Lw[c], P[(size_t)(E.ncomp + c) * TGT_TILE]);
                }
            }
        }
    }
    double acc[17];
#pragma unroll
    for (int c = 0; c < 17; ++c) acc[c] = (double)H[c] + (double)Lw[c];
    const double f4pi = 0.079577471545947667884;  // 1/(4 pi)
    const EpilogueOut& o = E.o;
    const double u0 = acc[0] * f4pi, u1 = acc[1] * f4pi, u2 = acc[2] * f4pi;
    double J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (E.ncomp >= 14) {
        const double Sx = acc[3], Sy = acc[4], Sz = acc[5];
        const double Gzz = -(acc[6] + acc[10]);
        // J = ([S x] - 3 G') / (4 pi)
        J[0] = (-3.0 * acc[6]) * f4pi;
        J[1] = (-Sz - 3.0 * acc[7]) * f4pi;
        J[2] = (Sy - 3.0 * acc[8]) * f4pi;
        J[3] = (Sz - 3.0 * acc[9]) * f4pi;
        J[4] = (-3.0 * acc[10]) * f4pi;
        J[5] = (-Sx - 3.0 * acc[11]) * f4pi;
        J[6] = (-Sy - 3.0 * acc[12]) * f4pi;
        J[7] = (Sx - 3.0 * acc[13]) * f4pi;
        J[8] = (-3.0 * Gzz) * f4pi;
    }
    if (o.mode == 0) {
        o.u[i] = (float)u0;
        o.u[E.n + i] = (float)u1;
        o.u[2 * E.n + i] = (float)u2;
        if (o.grad_u)
            for (int c = 0; c < 9; ++c) o.grad_u[(size_t)c * E.n + i] = (float)J[c];
        if (o.check_finite) {
            check_finite(E.dev_err, u0 + u1 + u2);
            if (o.grad_u) check_finite(E.dev_err, J[0] + J[1] + J[2] + J[3] + J[4] + J[5] + J[6] + J[7] + J[8]);
        }
        return;
    }
    // Right-hand side of Eq. 4-5 for particle i.
    const float4 G4 = reinterpret_cast<const float4*>(o.str)[i];
    const double Gm[3] = {G4.x, G4.y, G4.z};
    // Vreman: alpha = J^T, beta = Delta^2 g with g = J J^T (symmetric), Delta = sigma, so
    // B_beta = Delta^4 B_g and alpha:alpha = trace g: nu_t = c_V Delta^2 sqrt(B_g / trace g).
    auto dot3 = [&](int p, int q) { return J[3 * p] * J[3 * q] + J[3 * p + 1] * J[3 * q + 1] + J[3 * p + 2] * J[3 * q + 2]; };
    const double g00 = dot3(0, 0), g11 = dot3(1, 1), g22 = dot3(2, 2);
    const double g01 = dot3(0, 1), g02 = dot3(0, 2), g12 = dot3(1, 2);
    const double aa = g00 + g11 + g22;
    const double B = g00 * g11 - g01 * g01 + g00 * g22 - g02 * g02 + g11 * g22 - g12 * g12;
    const double nut =
        (aa > 0.0 && B > 0.0) ? (double)o.c_v * ((double)o.sigma * (double)o.sigma) * sqrt(B / aa) : 0.0;
    double s[3];
    if (E.ncomp == 17) {  // transposed stretching accumulated per target
        s[0] = acc[14] * f4pi;
        s[1] = acc[15] * f4pi;
        s[2] = acc[16] * f4pi;
    } else {
        for (int a = 0; a < 3; ++a) {
            double v = 0.0;
            for (int c = 0; c < 3; ++c) v += o.classic ? J[3 * a + c] * Gm[c] : J[3 * c + a] * Gm[c];
            s[a] = v;
        }
    }
    o.dxdt[i] = (float)(u0 + o.uinf[0]);
    o.dxdt[E.n + i] = (float)(u1 + o.uinf[1]);
    o.dxdt[2 * E.n + i] = (float)(u2 + o.uinf[2]);
    o.dGdt[i] = (float)s[0];
    o.dGdt[E.n + i] = (float)s[1];
    o.dGdt[2 * E.n + i] = (float)s[2];
    o.nu_t[i] = (float)nut;
    if (o.check_finite) check_finite(E.dev_err, u0 + u1 + u2 + s[0] + s[1] + s[2] + nut);
}

// ---------------------------------------------------------------------------
// Particle strength exchange (Eq. 5's diffusion term):
//   p_i = (2/sigma^2) sum_j nu_ij (v_i Gamma_j - v_j Gamma_i) zeta_sigma(r_ij),
//   nu_ij = nu + (nu_t,i + nu_t,j)/2, zeta of Eq. 3.
// Each warp owns 64 consecutive particles (two per lane) with two bounding boxes
// (split at the largest index-order jump).  It walks the source tiles 32 at a
// time, one box test per lane, and for every tile within 7 sigma of either box
// stages the tile (positions, strengths, nu_t) in its own slice of shared memory
// with coalesced loads, then every lane sums over it.  No block-wide barrier:
// warps proceed independently.  v_i Gamma_j - v_j Gamma_i is formed from two
// rounded products so that the i == j term is exactly zero; pairs beyond 7 sigma
// get exp(-r^2/2s^2) < 3e-11 and are skipped.
// ---------------------------------------------------------------------------
constexpr int PSE_T = 256;
constexpr int PSE_W = PSE_T / 32;

__device__ __forceinline__ void pse_pair(float4 pi, float4 gi, float base, float4 pj, float4 gj, float ntj,
                                         float inv2s2, float cut2, float& ax, float& ay, float& az)
{
    const float rx = pi.x - pj.x, ry = pi.y - pj.y, rz = pi.z - pj.z;
    const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
    if (r2 < cut2) {
        const float w = fmaf(0.5f, ntj, base) * expf(-r2 * inv2s2);
        const float vi = pi.w, vj = pj.w;
        ax = fmaf(w, __fsub_rn(__fmul_rn(vi, gj.x), __fmul_rn(vj, gi.x)), ax);
        ay = fmaf(w, __fsub_rn(__fmul_rn(vi, gj.y), __fmul_rn(vj, gi.y)), ay);
        az = fmaf(w, __fsub_rn(__fmul_rn(vi, gj.z), __fmul_rn(vj, gi.z)), az);
    }
}

__global__ void __launch_bounds__(PSE_T) pse_kernel(const float4* __restrict__ pos, const float4* __restrict__ str,
                                                    const float* __restrict__ nu_t, int n,
                                                    const float4* __restrict__ box, int ntiles, float inv2s2,
                                                    float cut2, float nu, float pref, float* __restrict__ dGdt)
{
    __shared__ float4 sp[PSE_W][SRC_TILE], sg[PSE_W][SRC_TILE];
    __shared__ float snt[PSE_W][SRC_TILE];
    __shared__ float wbox[PSE_W][12];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base_i = (blockIdx.x * PSE_W + warp) * 64;
    if (base_i >= n) return;  // whole warp past the end
    const int i0 = base_i + lane, i1 = i0 + 32;
    const bool v0 = i0 < n, v1 = i1 < n;
    float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0, g0 = p0, g1 = p0;
    float nt0 = 0.f, nt1 = 0.f;
    if (v0) p0 = pos[i0], g0 = str[i0], nt0 = nu_t ? nu_t[i0] : 0.f;
    if (v1) p1 = pos[i1], g1 = str[i1], nt1 = nu_t ? nu_t[i1] : 0.f;
    warp_two_boxes(make_float3(p0.x, p0.y, p0.z), v0, make_float3(p1.x, p1.y, p1.z), v1, wbox[warp]);
    const float base0 = nu + 0.5f * nt0, base1 = nu + 0.5f * nt1;
    float a0x = 0.f, a0y = 0.f, a0z = 0.f, a1x = 0.f, a1y = 0.f, a1z = 0.f;
    for (int tb = 0; tb < ntiles; tb += 32) {
        const int tt = tb + lane;
        const bool near = tt < ntiles && boxes_near(wbox[warp], box[2 * tt], box[2 * tt + 1], cut2);
        unsigned mask = __ballot_sync(0xffffffffu, near);
        while (mask) {
            const int tile = tb + __ffs(mask) - 1;
            mask &= mask - 1;
            const int j0 = tile * SRC_TILE, cnt = min(SRC_TILE, n - j0);
            // stage the tile; a source at least 7 sigma from both of the warp's target boxes
            // reaches none of its targets and is left out (warp-uniformly, by ballot)
            __syncwarp();
            unsigned keep[SRC_TILE / 32];
#pragma unroll
            for (int h = 0; h < SRC_TILE / 32; ++h) {
                const int q = lane + 32 * h;
                bool kp = false;
                if (q < cnt) {
                    const float4 pq = pos[j0 + q];
                    sp[warp][q] = pq;
                    sg[warp][q] = str[j0 + q];
                    snt[warp][q] = nu_t ? nu_t[j0 + q] : 0.f;
                    const float4 pt = make_float4(pq.x, pq.y, pq.z, 0.f);
                    kp = boxes_near(wbox[warp], pt, pt, cut2);
                }
                keep[h] = __ballot_sync(0xffffffffu, kp);
            }
            __syncwarp();
#pragma unroll
            for (int h = 0; h < SRC_TILE / 32; ++h)
            for (unsigned m = keep[h]; m; m &= m - 1) {
                const int j = 32 * h + __ffs(m) - 1;
                const float4 pj = sp[warp][j], gj = sg[warp][j];
                const float ntj = snt[warp][j];
                pse_pair(p0, g0, base0, pj, gj, ntj, inv2s2, cut2, a0x, a0y, a0z);
                pse_pair(p1, g1, base1, pj, gj, ntj, inv2s2, cut2, a1x, a1y, a1z);
            }
        }
    }
    if (v0) {
        dGdt[i0] += pref * a0x;
        dGdt[n + i0] += pref * a0y;
        dGdt[2 * n + i0] += pref * a0z;
    }
    if (v1) {
        dGdt[i1] += pref * a1x;
        dGdt[n + i1] += pref * a1y;
        dGdt[2 * n + i1] += pref * a1z;
    }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
__device__ int g_dev_err;  // device error word (one instance per device)

namespace {
std::mutex g_mu;
int g_sm[64];
int g_blocks[64][16];
bool g_attr[64][16];
}  // namespace

static int cur_dev()
{
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

int sm_count()
{
    const int d = cur_dev();
    std::lock_guard<std::mutex> lk(g_mu);
    if (d < 0 || d >= 64) return 0;
    if (!g_sm[d]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) v = 0;
        g_sm[d] = v;
    }
    return g_sm[d];
}

// The device error word of the current device, looked up on every call (a cheap
// query once the module is loaded) so that the address is never stale.
int* dev_err_ptr()
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dev_err) != cudaSuccess) return nullptr;
    return static_cast<int*>(p);
}

static int variant(bool G, bool C, bool S, int K) { return 8 * K + (G ? 4 : 0) + (C ? 2 : 0) + (S ? 1 : 0); }

// Opts the kernel into its dynamic shared memory (once per device) and returns the resident blocks per SM.
template <bool G, bool C, bool S, int K>
static int prepare_kernel(int d)
{
    const int v = variant(G, C, S, K);
    const size_t smem = sweep_smem_bytes<G, C, S>();
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (d >= 0 && d < 64 && g_attr[d][v]) return g_blocks[d][v];
    }
    cudaFuncSetAttribute(sweep_kernel<G, C, S, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<G, C, S, K>, SWEEP_TPB, smem) != cudaSuccess)
        nb = 1;
    if (nb < 1) nb = 1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (d >= 0 && d < 64) {
        g_blocks[d][v] = nb;
        g_attr[d][v] = true;
    }
    return nb;
}

template <int K>
static int blocks_per_sm_kind(bool g, bool c, bool s)
{
    const int d = cur_dev();
    if (g && s) return c ? prepare_kernel<true, true, true, K>(d) : prepare_kernel<true, false, true, K>(d);
    if (g) return c ? prepare_kernel<true, true, false, K>(d) : prepare_kernel<true, false, false, K>(d);
    return c ? prepare_kernel<false, true, false, K>(d) : prepare_kernel<false, false, false, K>(d);
}

static int blocks_per_sm(bool g, bool c, bool s, bool segments)
{
    return segments ? blocks_per_sm_kind<SWEEP_SEGMENTS>(g, c, s) : blocks_per_sm_kind<SWEEP_PARTICLES>(g, c, s);
}

int sweep_blocks(bool grad, bool comp, bool stretch, bool segments)
{
    const int sms = sm_count();
    return blocks_per_sm(grad, comp, stretch && grad, segments) * (sms > 0 ? sms : 1);
}

SweepPlan plan_sweep(int64_t n_tgt, int64_t n_src, int64_t m_seg, bool grad, bool comp, Carve& cv, bool stretch)
{
    SweepPlan p;
    p.n_tgt = (int)n_tgt;
    p.n_src = (int)n_src;
    p.m_seg = (int)m_seg;
    p.grad = grad;
    p.comp = comp;
    p.stretch = stretch && grad;
    p.ncomp = grad ? (p.stretch ? 17 : 14) : 3;
    p.TT = (int)((n_tgt + TGT_TILE - 1) / TGT_TILE);
    p.SP = (int)((n_src + SRC_TILE - 1) / SRC_TILE);
    p.SS = (int)((m_seg + SRC_TILE - 1) / SRC_TILE);
    // particle tiles and segment tiles: one stream-K plan (and launch) each
    auto plan = [&](StreamK& sk, int np, int ns) {
        sk.TT = p.TT;
        sk.np = np;
        sk.ns = ns;
        sk.wp = UNIT_W_P;
        sk.ws = grad ? UNIT_W_S_GRAD : UNIT_W_S_VEL;
        sk.C = (long long)sk.np * sk.wp + (long long)sk.ns * sk.ws;
        sk.tot = (long long)sk.TT * sk.C;
        const long long units = (long long)sk.TT * (sk.np + sk.ns);
        long long B = sweep_blocks(grad, comp, p.stretch, ns > 0);
        if (B > units) B = units;
        if (B < 1) B = 1;
        sk.B = (int)B;
    };
    // A small problem (fewer cost units than four waves of resident blocks) sweeps both
    // kinds of tile in one launch; a larger one gives the segment tiles a launch of
    // their own, where closed rings are packed by corner.
    const long long units_all = (long long)p.TT * (p.SP + p.SS);
    p.mixed = p.SP > 0 && p.SS > 0 && units_all < 4LL * sweep_blocks(grad, comp, p.stretch, false);
    plan(p.sk, p.SP, p.mixed ? p.SS : 0);
    plan(p.sks, 0, p.mixed ? 0 : p.SS);
    p.off_psrc = cv.take((size_t)p.SP * SRC_TILE * P_F4 * 16);
    p.off_pbox = cv.take((size_t)p.SP * 2 * 16);
    p.off_ssrc = cv.take((size_t)p.SS * SRC_TILE * S_F4 * 16);
    p.off_sbox = cv.take((size_t)p.SS * 2 * 16);
    const size_t rows = (size_t)(comp ? 2 : 1) * p.ncomp;
    if (p.sk.np + p.sk.ns > 0) p.off_part = cv.take((size_t)(p.sk.TT + p.sk.B) * rows * TGT_TILE * sizeof(float));
    if (p.sks.ns > 0) p.off_part_s = cv.take((size_t)(p.sks.TT + p.sks.B) * rows * TGT_TILE * sizeof(float));
    p.bytes = cv.off;
    return p;
}

template <bool G, bool C, bool S>
static void launch_sweep(const SweepArgs& A, int B, bool segments, cudaStream_t st)
{
    if (segments)
        sweep_kernel<G, C, S, SWEEP_SEGMENTS><<<B, SWEEP_TPB, sweep_smem_bytes<G, C, S>(), st>>>(A);
    else
        sweep_kernel<G, C, S, SWEEP_PARTICLES><<<B, SWEEP_TPB, sweep_smem_bytes<G, C, S>(), st>>>(A);
}

cudaError_t run_sweep(const SweepPlan& p, char* ws, const float* tgt, const float* src_pos, const float* src_str,
                      const float* seg_a, const float* seg_b, float sigma, float seg_core, int vatistas_n,
                      const EpilogueOut& out, cudaStream_t st)
{
    if (p.n_tgt == 0) return cudaSuccess;
    float4* psrc = reinterpret_cast<float4*>(ws + p.off_psrc);
    float4* pbox = reinterpret_cast<float4*>(ws + p.off_pbox);
    float4* ssrc = reinterpret_cast<float4*>(ws + p.off_ssrc);
    float4* sbox = reinterpret_cast<float4*>(ws + p.off_sbox);
    float* part = reinterpret_cast<float*>(ws + p.off_part);
    float* part_s = reinterpret_cast<float*>(ws + p.off_part_s);
    if (p.SP > 0) {
        trace_launch();
        pack_particles_kernel<<<p.SP, SRC_TILE, 0, st>>>(reinterpret_cast<const float4*>(src_pos),
                                                         reinterpret_cast<const float4*>(src_str), p.n_src, psrc,
                                                         pbox);
    }
    if (p.SS > 0) {
        trace_launch();
        pack_segments_kernel<<<p.SS, SRC_TILE, 0, st>>>(reinterpret_cast<const float4*>(seg_a),
                                                        reinterpret_cast<const float4*>(seg_b), p.m_seg, seg_core,
                                                        vatistas_n, p.mixed ? 0 : 1, ssrc, sbox);
    }
    int* err = dev_err_ptr();
    if (p.SP + p.SS > 0) {
        if (p.sk.np + p.sk.ns > 0) blocks_per_sm(p.grad, p.comp, p.stretch, false);  // shared-memory opt-in
        if (p.sks.ns > 0) blocks_per_sm(p.grad, p.comp, p.stretch, true);
        SweepArgs A;
        A.tgt = reinterpret_cast<const float4*>(tgt);
        A.tstr = p.stretch ? reinterpret_cast<const float4*>(out.str) : nullptr;
        A.n_tgt = p.n_tgt;
        A.psrc = psrc;
        A.pbox = pbox;
        A.n_src = p.n_src;
        A.ssrc = ssrc;
        A.sbox = sbox;
        A.core_pos = seg_core > 0.f ? 1 : 0;
        A.m_seg = p.m_seg;
        A.vn = vatistas_n;
        A.sk = p.sk;
        const double s = sigma;
        A.nc.inv_s2 = (float)(1.0 / (s * s));
        A.nc.inv_s3 = (float)(1.0 / (s * s * s));
        A.nc.inv_s5 = (float)(1.0 / (s * s * s * s * s));
        A.nc.far2 = (float)((double)RHO_FAR * RHO_FAR * s * s);
        A.dev_err = err;
        for (int kind = 0; kind < 2; ++kind) {
            const bool seg = kind == 1;
            if ((seg ? p.sks.ns : p.sk.np + p.sk.ns) == 0) continue;
            TraceScope ts(seg ? VPM_TRACE_SEGMENTS : p.grad ? VPM_TRACE_SWEEP : VPM_TRACE_SWEEP_VEL, st);
            A.sk = seg ? p.sks : p.sk;
            A.part = seg ? part_s : part;
            const int B = A.sk.B;
            if (p.grad && p.stretch) {
                if (p.comp)
                    launch_sweep<true, true, true>(A, B, seg, st);
                else
                    launch_sweep<true, false, true>(A, B, seg, st);
            } else if (p.grad) {
                if (p.comp)
                    launch_sweep<true, true, false>(A, B, seg, st);
                else
                    launch_sweep<true, false, false>(A, B, seg, st);
            } else {
                if (p.comp)
                    launch_sweep<false, true, false>(A, B, seg, st);
                else
                    launch_sweep<false, false, false>(A, B, seg, st);
            }
        }
    }
    EpiArgs E;
    E.sk = p.sk;
    E.part = part;
    E.sks = p.sks;
    E.part_s = part_s;
    E.n = p.n_tgt;
    E.ncomp = p.ncomp;
    E.comp = p.comp ? 1 : 0;
    E.o = out;
    E.dev_err = err;
    trace_launch();
    epilogue_kernel<<<(p.n_tgt + 255) / 256, 256, 0, st>>>(E);
    return cudaGetLastError();
}

cudaError_t run_pse(const SweepPlan& p, char* ws, const float* pos, const float* str, const float* nu_t, int n,
                    float sigma, float nu, float* dGdt, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const float4* pbox = reinterpret_cast<const float4*>(ws + p.off_pbox);
    const double s = sigma;
    const float inv2s2 = (float)(0.5 / (s * s));
    const float cut2 = (float)((double)RHO_FAR * RHO_FAR * s * s);
    // (2/sigma^2) (2 pi sigma^2)^(-3/2)
    const float pref = (float)(2.0 / (s * s) * pow(2.0 * 3.14159265358979323846 * s * s, -1.5));
    TraceScope ts(VPM_TRACE_PSE, st);
    pse_kernel<<<(n + 64 * PSE_W - 1) / (64 * PSE_W), PSE_T, 0, st>>>(reinterpret_cast<const float4*>(pos),
                                                          reinterpret_cast<const float4*>(str), nu_t, n, pbox, p.SP,
                                                          inv2s2, cut2, nu, pref, dGdt);
    return cudaGetLastError();
}

}  // namespace vpm
