// Near-field Gaussian blob kernel shared by the forward and adjoint pair sweeps.
#pragma once

#include <cuda_runtime.h>

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

}  // namespace vpm
