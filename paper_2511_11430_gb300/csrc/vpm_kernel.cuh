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

}  // namespace vpm
