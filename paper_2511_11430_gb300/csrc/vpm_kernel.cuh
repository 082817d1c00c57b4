// Gaussian blob kernel and per-pair accumulation shared by the pair sweeps, the
// adjoint and the treecode.
#pragma once

#include <cuda_runtime.h>

#include "vpm_common.cuh"

namespace vpm {

// ---------------------------------------------------------------------------
// Regularised blob kernel, near field.
//
// With x = rho^2/2 the enclosed-vorticity fraction of Eq. 3's Gaussian is the
// regularised lower incomplete gamma function g = P(3/2, x), and its series
//   P(3/2, x) = x^(3/2) e^(-x) sum_k x^k / Gamma(k + 5/2)
// has only positive terms.  Hence, with K = q(rho)/(4 pi sigma^3) and
// H = f(rho)/(4 pi sigma^5),
//   q = g / rho^3      =  2^(-3/2) e^(-x) sum_k x^k / Gamma(k + 5/2)
//   f = q'(rho) / rho  = dq/dx = -(3/2) 2^(-3/2) e^(-x) sum_k x^k / Gamma(k + 7/2)
// (the second by differentiating the first term by term: the x^k coefficient of
// T' - T, T the sum in q, is ((k + 1) - (k + 5/2)) / Gamma(k + 7/2)), both free of
// cancellation.  For x >= 2 the closed form g = erf(sqrt x) - sqrt(2/pi) rho e^(-x)
// loses at most a factor 1.3 and is used instead.
// ---------------------------------------------------------------------------
struct SeriesCoef {
    float c[16];  // 1 / Gamma(k + 5/2)
    float d[16];  // (3/2) / Gamma(k + 7/2)
};

constexpr SeriesCoef make_series()
{
    SeriesCoef s{};
    double ck = 0.75225277806367504925;  // 1/Gamma(5/2) = 4/(3 sqrt(pi))
    for (int k = 0; k < 16; ++k) {
        s.c[k] = (float)ck;
        const double cn = ck / (k + 2.5);  // 1/Gamma(k + 7/2)
        s.d[k] = (float)(1.5 * cn);
        ck = cn;
    }
    return s;
}

static __constant__ SeriesCoef kSeries = make_series();

struct NearConst {
    float inv_s2, inv_s3, inv_s5, far2;
};

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x of both lanes of a packed pair.
__device__ __forceinline__ float2 rcp2_approx(float2 x)
{
    unsigned long long in = *reinterpret_cast<unsigned long long*>(&x), out;
    asm("{\n\t.reg .f32 a, b;\n\t"
        "mov.b64 {a, b}, %1;\n\t"
        "rcp.approx.ftz.f32 a, a;\n\t"
        "rcp.approx.ftz.f32 b, b;\n\t"
        "mov.b64 %0, {a, b};\n\t}"
        : "=l"(out)
        : "l"(in));
    return *reinterpret_cast<float2*>(&out);
}

// rsqrt of both lanes of a packed pair, produced directly into a register pair.
__device__ __forceinline__ float2 rsqrt2_approx(float2 x)
{
    unsigned long long in = *reinterpret_cast<unsigned long long*>(&x), out;
    asm("{\n\t.reg .f32 a, b;\n\t"
        "mov.b64 {a, b}, %1;\n\t"
        "rsqrt.approx.ftz.f32 a, a;\n\t"
        "rsqrt.approx.ftz.f32 b, b;\n\t"
        "mov.b64 %0, {a, b};\n\t}"
        : "=l"(out)
        : "l"(in));
    return *reinterpret_cast<float2*>(&out);
}

// K (without 1/(4 pi)) and h = H * (-1/3) (without 1/(4 pi)) of one pair; in the far
// field K = r^-3 and h = r^-5.  A pair at zero distance contributes nothing.
__device__ __forceinline__ void near_kh(float r2, const NearConst& nc, float& K, float& h)
{
    if (r2 == 0.f) {
        K = 0.f;
        h = 0.f;
        return;
    }
    if (r2 >= nc.far2) {
        const float rs = rsqrt_approx(r2);
        const float i2 = rs * rs;
        K = i2 * rs;
        h = K * i2;
        return;
    }
    const float x = 0.5f * r2 * nc.inv_s2;
    float q, f;
    if (x < 2.0f) {
        float T = kSeries.c[15], U = kSeries.d[15];
#pragma unroll
        for (int k = 14; k >= 0; --k) {
            T = fmaf(T, x, kSeries.c[k]);
            U = fmaf(U, x, kSeries.d[k]);
        }
        const float e = expf(-x) * 0.35355339059327376f;  // 2^(-3/2) e^(-x)
        q = e * T;
        f = -e * U;
    } else {
        const float rho2 = 2.0f * x;
        const float rho = sqrtf(rho2);
        const float e = expf(-x);
        const float g = erff(sqrtf(x)) - 0.79788456080286536f * rho * e;
        q = g / (rho * rho2);
        f = (0.79788456080286536f * e - 3.0f * q) / rho2;
    }
    K = q * nc.inv_s3;
    h = f * (-1.0f / 3.0f) * nc.inv_s5;
}

// ---------------------------------------------------------------------------
// Accumulators of one thread (two targets per f2): u, S, the 8 independent
// entries of G' = sum h (Gamma x r) (x) r (its trace vanishes pair by pair, so
// G'_zz = -G'_xx - G'_yy) and, with STRETCH, s = 4 pi J^T Gamma_i.
// J = ([S x] - 3 G') / (4 pi), u = u / (4 pi).
// ---------------------------------------------------------------------------
template <bool GRAD, bool STRETCH>
struct Acc {
    static constexpr int N = GRAD ? (STRETCH ? 17 : 14) : 3;
    f2 v[N];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = zero2();
    }
};

// The target's own strength, for the stretching terms.
struct Own {
    f2 gx, gy, gz;
};

template <bool GRAD, bool STRETCH, bool NEAR>
__device__ __forceinline__ void accum_particle(Acc<GRAD, STRETCH>& a, f2 K, f2 h, f2 rx, f2 ry, f2 rz, f2 gx, f2 gy,
                                               f2 gz, f2 ngx, f2 ngy, f2 ngz, const Own& o)
{
    const f2 cx = fma2(gy, rz, mul2(ngz, ry));
    const f2 cy = fma2(gz, rx, mul2(ngx, rz));
    const f2 cz = fma2(gx, ry, mul2(ngy, rx));
    a.v[0] = fma2(K, cx, a.v[0]);
    a.v[1] = fma2(K, cy, a.v[1]);
    a.v[2] = fma2(K, cz, a.v[2]);
    if (GRAD) {
        a.v[3] = fma2(K, gx, a.v[3]);
        a.v[4] = fma2(K, gy, a.v[4]);
        a.v[5] = fma2(K, gz, a.v[5]);
        const f2 hx = mul2(h, cx), hy = mul2(h, cy), hz = mul2(h, cz);
        a.v[6] = fma2(hx, rx, a.v[6]);
        a.v[7] = fma2(hx, ry, a.v[7]);
        a.v[8] = fma2(hx, rz, a.v[8]);
        a.v[9] = fma2(hy, rx, a.v[9]);
        a.v[10] = fma2(hy, ry, a.v[10]);
        a.v[11] = fma2(hy, rz, a.v[11]);
        a.v[12] = fma2(hz, rx, a.v[12]);
        a.v[13] = fma2(hz, ry, a.v[13]);
    }
    if (STRETCH && NEAR) {
        // Transposed stretching per pair, written with d = Gamma_j - Gamma_i (exact
        // when the strengths are close) so that nothing cancels:
        //   K (Gamma_i x Gamma_j) = K (Gamma_i x d),
        //   -3 h ((Gamma_j x r) . Gamma_i) r = 3 h (d . (Gamma_i x r)) r.
        const f2 dx = sub2(gx, o.gx), dy = sub2(gy, o.gy), dz = sub2(gz, o.gz);
        const f2 tx = sub2(mul2(o.gy, dz), mul2(o.gz, dy));
        const f2 ty = sub2(mul2(o.gz, dx), mul2(o.gx, dz));
        const f2 tz = sub2(mul2(o.gx, dy), mul2(o.gy, dx));
        a.v[14] = fma2(K, tx, a.v[14]);
        a.v[15] = fma2(K, ty, a.v[15]);
        a.v[16] = fma2(K, tz, a.v[16]);
        const f2 ex = sub2(mul2(o.gy, rz), mul2(o.gz, ry));
        const f2 ey = sub2(mul2(o.gz, rx), mul2(o.gx, rz));
        const f2 ez = sub2(mul2(o.gx, ry), mul2(o.gy, rx));
        const f2 w = mul2(mul2(h, splat(3.f)), fma2(dz, ez, fma2(dy, ey, mul2(dx, ex))));
        a.v[14] = fma2(w, rx, a.v[14]);
        a.v[15] = fma2(w, ry, a.v[15]);
        a.v[16] = fma2(w, rz, a.v[16]);
    }
}

// Packed particle source (5 float4, both lanes equal):
//   (-x,-x,-y,-y) (-z,-z,gx,gx) (gy,gy,gz,gz) (-gx,-gx,-gy,-gy) (-gz,-gz,0,0)
// One source of a particle tile against the thread's two targets.
template <bool GRAD, bool STRETCH, bool NEAR>
__device__ __forceinline__ void particle_source(Acc<GRAD, STRETCH>& a, const float4* __restrict__ e, f2 X, f2 Y,
                                                f2 Z, const NearConst& nc, const Own& o)
{
    const float4 q0 = e[0], q1 = e[1], q2 = e[2], q3 = e[3], q4 = e[4];
    const f2 rx = add2(X, make_float2(q0.x, q0.y));
    const f2 ry = add2(Y, make_float2(q0.z, q0.w));
    const f2 rz = add2(Z, make_float2(q1.x, q1.y));
    const f2 r2 = fma2(rz, rz, fma2(ry, ry, mul2(rx, rx)));
    f2 K, h;
    if (NEAR) {
        near_kh(r2.x, nc, K.x, h.x);
        near_kh(r2.y, nc, K.y, h.y);
    } else {
        const f2 rs = rsqrt2_approx(r2);
        const f2 i2 = mul2(rs, rs);
        K = mul2(i2, rs);
        h = GRAD ? mul2(K, i2) : K;
    }
    accum_particle<GRAD, STRETCH, NEAR>(a, K, h, rx, ry, rz, make_float2(q1.z, q1.w), make_float2(q2.x, q2.y),
                                        make_float2(q2.z, q2.w), make_float2(q3.x, q3.y),
                                        make_float2(q3.z, q3.w), make_float2(q4.x, q4.y), o);
}

// ---------------------------------------------------------------------------
// Vatistas-cored straight segments (Sec. II.A) against two packed targets.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Inverse lengths of one segment pair for one lane, with the end-point and axis
// guards: a target within 1e-10 |r0| (or 1e-15 m) of an end point, or with
// D == 0, gets zero (all outputs zero so every later product stays finite).
__device__ __forceinline__ void seg_lane(float n1, float n2, float c2, float L2, float e, int vn, float& i1,
                                         float& i2, float& irs, float& invD)
{
    const float thr = fmaxf(1e-20f * L2, 1e-30f);  // (1e-10 |r0|)^2, (1e-15 m)^2
    const bool ok = (n1 > thr) && (n2 > thr);
    float D;
    if (vn == 2) {
        D = fmaf(c2, c2, e);
        invD = D > 0.f ? rsqrt_approx(D) : 0.f;
    } else {
        D = c2 + e;
        invD = D > 0.f ? __frcp_rn(D) : 0.f;
    }
    if (!ok || !(D > 0.f)) {
        i1 = i2 = irs = invD = 0.f;
        return;
    }
    i1 = rsqrt_approx(n1);
    i2 = rsqrt_approx(n2);
    irs = rcp_approx(fmaf(n1, i1, n2 * i2));  // 1 / (|r1| + |r2|)
}

// Packed segment source (6 float4, both lanes equal):
//   (-ax,-ax,-ay,-ay) (-az,-az,r0x,r0x) (r0y,r0y,r0z,r0z) (-r0x,-r0x,-r0y,-r0y) (-r0z,-r0z,-L2,-L2) (G,G,e,e)
// with r0 = b - a, L2 = |r0|^2, e = (core |r0|)^(2n).  With r1 = x - a, r2 = x - b,
// c = r0 x r1 (= r1 x r2), D = (|c|^(2n) + e)^(1/n):
//   u = G/(4 pi) c d / D,   d = r0 . (r1/|r1| - r2/|r2|),
//   J = G/(4 pi D) ( d [r0 x] + c (x) w ),   w = grad d - d grad D / D.
// Both are written to avoid cancellation in FP32:
//   d = (r0 . r1) (1/|r1| - 1/|r2|) + L2/|r2|,
//     1/|r1| - 1/|r2| = (L2 - 2 r0.r1) / (|r1| |r2| (|r1| + |r2|))   (|r2|^2 - |r1|^2 = L2 - 2 r0.r1),
//   grad d = (r1/|r1|^3 - r2/|r2|^3) x c   (the projections of r0 normal to r1, r2),
//   grad D / D = 2 |c|^(2n-2) D^(-n) (c x r0),   so  w = (r1/|r1|^3 - r2/|r2|^3 + k3 r0) x c
//   with k3 = 2 d |c|^(2n-2) D^(-n).
// SAFE: the warp's targets are at least 1e-3 of the longest segment away from the
// tile's bounding box and the core is positive, so no guard can trigger and every
// reciprocal is taken on both lanes at once.
// One segment (r0 = b - a and its negation, L2 = |r0|^2, e, circulation gs) against
// the thread's two targets at r1 = x - a, r2 = x - b.
template <bool GRAD, bool STRETCH, bool SAFE>
__device__ __forceinline__ void segment_pair(Acc<GRAD, STRETCH>& a, f2 r0x, f2 r0y, f2 r0z, f2 nr0x, f2 nr0y, f2 nr0z,
                                             f2 L2, f2 e, f2 gs, f2 r1x, f2 r1y, f2 r1z, f2 r2x, f2 r2y, f2 r2z, int vn)
{
    {
        const f2 cx = fma2(r0y, r1z, mul2(nr0z, r1y));
        const f2 cy = fma2(r0z, r1x, mul2(nr0x, r1z));
        const f2 cz = fma2(r0x, r1y, mul2(nr0y, r1x));
        const f2 n1 = fma2(r1z, r1z, fma2(r1y, r1y, mul2(r1x, r1x)));
        const f2 n2 = fma2(r2z, r2z, fma2(r2y, r2y, mul2(r2x, r2x)));
        const f2 p1 = fma2(r0z, r1z, fma2(r0y, r1y, mul2(r0x, r1x)));
        const f2 c2 = fma2(cz, cz, fma2(cy, cy, mul2(cx, cx)));
        f2 i1, i2, irs, invD;
        if (SAFE) {
            i1 = rsqrt2_approx(n1);
            i2 = rsqrt2_approx(n2);
            invD = vn == 2 ? rsqrt2_approx(fma2(c2, c2, e)) : rcp2_approx(add2(c2, e));
            irs = rcp2_approx(fma2(n1, i1, mul2(n2, i2)));
        } else {
            seg_lane(n1.x, n2.x, c2.x, L2.x, e.x, vn, i1.x, i2.x, irs.x, invD.x);
            seg_lane(n1.y, n2.y, c2.y, L2.y, e.y, vn, i1.y, i2.y, irs.y, invD.y);
        }
        const f2 di = mul2(mul2(fma2(splat(-2.f), p1, L2), mul2(i1, i2)), irs);  // 1/|r1| - 1/|r2|
        const f2 d = fma2(p1, di, mul2(L2, i2));
        const f2 gi = mul2(gs, invD);
        const f2 coef = mul2(gi, d);
        a.v[0] = fma2(coef, cx, a.v[0]);
        a.v[1] = fma2(coef, cy, a.v[1]);
        a.v[2] = fma2(coef, cz, a.v[2]);
        if (GRAD) {
            a.v[3] = fma2(coef, r0x, a.v[3]);
            a.v[4] = fma2(coef, r0y, a.v[4]);
            a.v[5] = fma2(coef, r0z, a.v[5]);
            f2 k3;
            if (vn == 2) {
                const f2 tmp = mul2(mul2(d, c2), mul2(invD, invD));
                k3 = add2(tmp, tmp);
            } else {
                const f2 tmp = mul2(d, invD);
                k3 = add2(tmp, tmp);
            }
            const f2 i1c = mul2(mul2(i1, i1), i1);
            const f2 ni2c = mul2(mul2(i2, i2), mul2(i2, splat(-1.f)));
            const f2 vx = fma2(k3, r0x, fma2(r1x, i1c, mul2(r2x, ni2c)));
            const f2 vy = fma2(k3, r0y, fma2(r1y, i1c, mul2(r2y, ni2c)));
            const f2 vz = fma2(k3, r0z, fma2(r1z, i1c, mul2(r2z, ni2c)));
            const f2 nvx = mul2(vx, splat(-1.f)), nvy = mul2(vy, splat(-1.f)), nvz = mul2(vz, splat(-1.f));
            const f2 wx = fma2(vy, cz, mul2(nvz, cy));  // w = v x c
            const f2 wy = fma2(vz, cx, mul2(nvx, cz));
            const f2 wz = fma2(vx, cy, mul2(nvy, cx));
            const f2 cg = mul2(gi, splat(-1.0f / 3.0f));  // stored as G' with J = -3 G'
            const f2 gx = mul2(cg, cx), gy = mul2(cg, cy), gz = mul2(cg, cz);
            a.v[6] = fma2(gx, wx, a.v[6]);
            a.v[7] = fma2(gx, wy, a.v[7]);
            a.v[8] = fma2(gx, wz, a.v[8]);
            a.v[9] = fma2(gy, wx, a.v[9]);
            a.v[10] = fma2(gy, wy, a.v[10]);
            a.v[11] = fma2(gy, wz, a.v[11]);
            a.v[12] = fma2(gz, wx, a.v[12]);
            a.v[13] = fma2(gz, wy, a.v[13]);
        }
    }
}

template <bool GRAD, bool STRETCH, bool SAFE>
__device__ __forceinline__ void segment_source(Acc<GRAD, STRETCH>& a, const float4* __restrict__ e4, f2 X, f2 Y, f2 Z,
                                               int vn)
{
    const float4 s0 = e4[0], s1 = e4[1], s2 = e4[2], s3 = e4[3], s4 = e4[4], s5 = e4[5];
    const f2 r0x = make_float2(s1.z, s1.w), r0y = make_float2(s2.x, s2.y), r0z = make_float2(s2.z, s2.w);
    const f2 nr0x = make_float2(s3.x, s3.y), nr0y = make_float2(s3.z, s3.w), nr0z = make_float2(s4.x, s4.y);
    const f2 L2 = mul2(make_float2(s4.z, s4.w), splat(-1.f));
    const f2 r1x = add2(X, make_float2(s0.x, s0.y));
    const f2 r1y = add2(Y, make_float2(s0.z, s0.w));
    const f2 r1z = add2(Z, make_float2(s1.x, s1.y));
    const f2 r2x = add2(r1x, nr0x), r2y = add2(r1y, nr0y), r2z = add2(r1z, nr0z);
    segment_pair<GRAD, STRETCH, SAFE>(a, r0x, r0y, r0z, nr0x, nr0y, nr0z, L2, make_float2(s5.z, s5.w),
                                      make_float2(s5.x, s5.y), r1x, r1y, r1z, r2x, r2y, r2z, vn);
}

// The sources of a segment tile (S_F4 float4 each) against the thread's two targets.
template <bool GRAD, bool STRETCH, bool SAFE>
__device__ __forceinline__ void segment_tile(Acc<GRAD, STRETCH>& a, const float4* __restrict__ s, int cnt, f2 X, f2 Y,
                                             f2 Z, int vn)
{
#pragma unroll 2
    for (int j = 0; j < cnt; ++j) segment_source<GRAD, STRETCH, SAFE>(a, s + j * S_F4, X, Y, Z, vn);
}

// ---------------------------------------------------------------------------
// Closed four-sided rings (the blade and wake vortex rings of Sec. II.A): side k runs
// from corner c_k to corner c_(k+1 mod 4), so side k's r2 = x - c_(k+1) is side k+1's r1.
// A tile whose segments all form such rings (in groups of four, bit-exact shared end
// points) is packed by ring, and each target evaluates x - c, |x - c|^2, 1/|x - c|,
// |x - c| and 1/|x - c|^3 once per corner instead of once per side end.  Packed ring
// (24 float4 = four segments' worth; pair p = floats 2p, 2p + 1, both lanes equal):
//   pairs  0..11  -c_k (k = 0..3; x, y, z)
//   pairs 12..23  r0_k = c_(k+1) - c_k        pairs 24..35  -r0_k
//   pairs 36..43  (L2_k, e_k)                 pairs 44..47  G_k
// The side terms are those of segment_source, with 1/|r1| - 1/|r2| formed as
// (L2 - 2 r0.r1) / (|r1| |r2| (|r1| + |r2|)) from one reciprocal.
// ---------------------------------------------------------------------------
template <int P>
__device__ __forceinline__ f2 ring_pair(const float4* __restrict__ e4)
{
    const float4 q = e4[P >> 1];
    return (P & 1) ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
}

struct RingCorner {
    f2 x, y, z;  // x - c
    f2 n;        // |x - c|^2
    f2 i;        // 1 / |x - c|
    f2 len;      // |x - c|
    f2 i3;       // 1 / |x - c|^3
};

template <int K>
__device__ __forceinline__ RingCorner ring_corner(const float4* __restrict__ e4, f2 X, f2 Y, f2 Z)
{
    RingCorner c;
    c.x = add2(X, ring_pair<3 * K>(e4));
    c.y = add2(Y, ring_pair<3 * K + 1>(e4));
    c.z = add2(Z, ring_pair<3 * K + 2>(e4));
    c.n = fma2(c.z, c.z, fma2(c.y, c.y, mul2(c.x, c.x)));
    c.i = rsqrt2_approx(c.n);
    c.len = mul2(c.n, c.i);
    c.i3 = mul2(mul2(c.i, c.i), c.i);
    return c;
}

// Side K of a ring between corners c1 = c_K and c2 = c_(K+1), for targets clear of the
// tile (no guard can trigger; as SAFE in segment_source).
template <bool GRAD, int K>
__device__ __forceinline__ void ring_side(Acc<GRAD, false>& a, const float4* __restrict__ e4, const RingCorner& c1,
                                          const RingCorner& c2, int vn)
{
    const f2 r0x = ring_pair<12 + 3 * K>(e4), r0y = ring_pair<13 + 3 * K>(e4), r0z = ring_pair<14 + 3 * K>(e4);
    const f2 nr0x = ring_pair<24 + 3 * K>(e4), nr0y = ring_pair<25 + 3 * K>(e4), nr0z = ring_pair<26 + 3 * K>(e4);
    const f2 L2 = ring_pair<36 + 2 * K>(e4), e = ring_pair<37 + 2 * K>(e4), gs = ring_pair<44 + K>(e4);
    const f2 r1x = c1.x, r1y = c1.y, r1z = c1.z;
    const f2 cx = fma2(r0y, r1z, mul2(nr0z, r1y));
    const f2 cy = fma2(r0z, r1x, mul2(nr0x, r1z));
    const f2 cz = fma2(r0x, r1y, mul2(nr0y, r1x));
    const f2 p1 = fma2(r0z, r1z, fma2(r0y, r1y, mul2(r0x, r1x)));
    const f2 c2n = fma2(cz, cz, fma2(cy, cy, mul2(cx, cx)));
    const f2 invD = vn == 2 ? rsqrt2_approx(fma2(c2n, c2n, e)) : rcp2_approx(add2(c2n, e));
    const f2 rP = rcp2_approx(mul2(mul2(c1.len, c2.len), add2(c1.len, c2.len)));
    const f2 i2 = c2.i, i1c = c1.i3, ni2c = mul2(c2.i3, splat(-1.f));
    const f2 di = mul2(fma2(splat(-2.f), p1, L2), rP);  // 1/|r1| - 1/|r2|
    const f2 d = fma2(p1, di, mul2(L2, i2));
    const f2 gi = mul2(gs, invD);
    const f2 coef = mul2(gi, d);
    a.v[0] = fma2(coef, cx, a.v[0]);
    a.v[1] = fma2(coef, cy, a.v[1]);
    a.v[2] = fma2(coef, cz, a.v[2]);
    if (GRAD) {
        a.v[3] = fma2(coef, r0x, a.v[3]);
        a.v[4] = fma2(coef, r0y, a.v[4]);
        a.v[5] = fma2(coef, r0z, a.v[5]);
        f2 k3;
        if (vn == 2) {
            const f2 tmp = mul2(mul2(d, c2n), mul2(invD, invD));
            k3 = add2(tmp, tmp);
        } else {
            const f2 tmp = mul2(d, invD);
            k3 = add2(tmp, tmp);
        }
        const f2 vx = fma2(k3, r0x, fma2(r1x, i1c, mul2(c2.x, ni2c)));
        const f2 vy = fma2(k3, r0y, fma2(r1y, i1c, mul2(c2.y, ni2c)));
        const f2 vz = fma2(k3, r0z, fma2(r1z, i1c, mul2(c2.z, ni2c)));
        const f2 nvx = mul2(vx, splat(-1.f)), nvy = mul2(vy, splat(-1.f)), nvz = mul2(vz, splat(-1.f));
        const f2 wx = fma2(vy, cz, mul2(nvz, cy));  // w = v x c
        const f2 wy = fma2(vz, cx, mul2(nvx, cz));
        const f2 wz = fma2(vx, cy, mul2(nvy, cx));
        const f2 cg = mul2(gi, splat(-1.0f / 3.0f));  // stored as G' with J = -3 G'
        const f2 gx = mul2(cg, cx), gy = mul2(cg, cy), gz = mul2(cg, cz);
        a.v[6] = fma2(gx, wx, a.v[6]);
        a.v[7] = fma2(gx, wy, a.v[7]);
        a.v[8] = fma2(gx, wz, a.v[8]);
        a.v[9] = fma2(gy, wx, a.v[9]);
        a.v[10] = fma2(gy, wy, a.v[10]);
        a.v[11] = fma2(gy, wz, a.v[11]);
        a.v[12] = fma2(gz, wx, a.v[12]);
        a.v[13] = fma2(gz, wy, a.v[13]);
    }
}

// The rings of a ring-packed segment tile (cnt rings, 4 S_F4 float4 each).  Targets
// close to the tile (SAFE false) take segment_pair's guarded form side by side, with
// r2 = x - c_(k+1) read from the next corner.
template <bool GRAD, bool SAFE>
__device__ __forceinline__ void ring_tile(Acc<GRAD, false>& a, const float4* __restrict__ s, int cnt, f2 X, f2 Y,
                                          f2 Z, int vn)
{
    if constexpr (SAFE) {
#pragma unroll 1
        for (int j = 0; j < cnt; ++j) {
            const float4* e4 = s + j * 4 * S_F4;
            const RingCorner c0 = ring_corner<0>(e4, X, Y, Z);
            const RingCorner c1 = ring_corner<1>(e4, X, Y, Z);
            ring_side<GRAD, 0>(a, e4, c0, c1, vn);
            const RingCorner c2 = ring_corner<2>(e4, X, Y, Z);
            ring_side<GRAD, 1>(a, e4, c1, c2, vn);
            const RingCorner c3 = ring_corner<3>(e4, X, Y, Z);
            ring_side<GRAD, 2>(a, e4, c2, c3, vn);
            ring_side<GRAD, 3>(a, e4, c3, c0, vn);
        }
    } else {
#pragma unroll 1
        for (int j = 0; j < cnt; ++j) {
            const float2* p = reinterpret_cast<const float2*>(s + j * 4 * S_F4);
#pragma unroll 1
            for (int k = 0; k < 4; ++k) {
                const int k1 = (k + 1) & 3;
                const f2 r1x = add2(X, p[3 * k]), r1y = add2(Y, p[3 * k + 1]), r1z = add2(Z, p[3 * k + 2]);
                const f2 r2x = add2(X, p[3 * k1]), r2y = add2(Y, p[3 * k1 + 1]), r2z = add2(Z, p[3 * k1 + 2]);
                segment_pair<GRAD, false, false>(a, p[12 + 3 * k], p[13 + 3 * k], p[14 + 3 * k], p[24 + 3 * k],
                                                 p[25 + 3 * k], p[26 + 3 * k], p[36 + 2 * k], p[37 + 2 * k],
                                                 p[44 + k], r1x, r1y, r1z, r2x, r2y, r2z, vn);
            }
        }
    }
}

}  // namespace vpm
