// Low-storage third-order Runge-Kutta step (Williamson 1980), the time update
// the paper applies to Eq. 4-5:
//   for k = 1..3:  q <- A_k q + dt f(y);  y <- y + B_k q,
//   A = (0, -5/9, -153/128),  B = (1/3, 15/16, 8/15).
// The state y = (x, Gamma) and the register q stay in FP64; the right-hand side
// f arrives in FP32 from the pair sweeps, and each stage writes the FP32 packed
// copy of y that the next right-hand side reads.  Pure streaming kernels: per
// particle and stage they move 6 doubles of y and of q in and out, 6 floats of f
// in and 8 floats of packed state out.
#include "vpm_internal.h"

namespace vpm {

__global__ void __launch_bounds__(256) cast_state_kernel(const double* __restrict__ x, const double* __restrict__ G,
                                                         const float* __restrict__ vol, int n,
                                                         float4* __restrict__ pos, float4* __restrict__ str)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pos[i] = make_float4((float)x[i], (float)x[n + i], (float)x[2 * n + i], vol[i]);
    str[i] = make_float4((float)G[i], (float)G[n + i], (float)G[2 * n + i], 0.f);
}

__global__ void __launch_bounds__(256) rk3_stage_kernel(int k, double dt, double* __restrict__ x,
                                                        double* __restrict__ G, double* __restrict__ qx,
                                                        double* __restrict__ qG, const float* __restrict__ fx,
                                                        const float* __restrict__ fG, const float* __restrict__ vol,
                                                        int n, float4* __restrict__ pos, float4* __restrict__ str)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double A = k == 0 ? 0.0 : (k == 1 ? -5.0 / 9.0 : -153.0 / 128.0);
    const double B = k == 0 ? 1.0 / 3.0 : (k == 1 ? 15.0 / 16.0 : 8.0 / 15.0);
    double y[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t o = (size_t)c * n + i;
        // first stage: q = dt f (A_1 = 0; q is not read, it may hold anything)
        const double q1 = (k == 0 ? 0.0 : A * qx[o]) + dt * (double)fx[o];
        const double q2 = (k == 0 ? 0.0 : A * qG[o]) + dt * (double)fG[o];
        qx[o] = q1;
        qG[o] = q2;
        y[c] = x[o] + B * q1;
        y[3 + c] = G[o] + B * q2;
        x[o] = y[c];
        G[o] = y[3 + c];
    }
    if (pos) {
        pos[i] = make_float4((float)y[0], (float)y[1], (float)y[2], vol[i]);
        str[i] = make_float4((float)y[3], (float)y[4], (float)y[5], 0.f);
    }
}

cudaError_t run_cast_state(const double* x, const double* G, const float* vol, int n, float* pos, float* str,
                           cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    trace_launch();
    cast_state_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, G, vol, n, reinterpret_cast<float4*>(pos),
                                                       reinterpret_cast<float4*>(str));
    return cudaGetLastError();
}

cudaError_t run_rk3_stage(int k, double dt, double* x, double* G, double* qx, double* qG, const float* dxdt,
                          const float* dGdt, const float* vol, int n, float* pos, float* str, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    trace_launch();
    rk3_stage_kernel<<<(n + 255) / 256, 256, 0, st>>>(k, dt, x, G, qx, qG, dxdt, dGdt, vol, n,
                                                      reinterpret_cast<float4*>(pos), reinterpret_cast<float4*>(str));
    return cudaGetLastError();
}

}  // namespace vpm
