// Blade loads of the vortex-lattice blades (Sec. II.A): the steady part by the
// Kutta-Joukowski theorem on every bound segment (panel side),
//   F_s = rho Gamma_s (V_s x (b_s - a_s)),  V_s = u_inf - omega x (mid_s - hub) + u_ind(mid_s),
// and the unsteady part at the centre of every panel (unsteady Bernoulli),
//   F_p = rho (Gamma_p - Gamma_p,prev) / dt  A_p n_p,
// with the total force and its moment about the hub.  The per-item terms are formed
// in FP64 and reduced by one block in a fixed order (deterministic).
#include "vpm_internal.h"

namespace vpm {

__device__ __forceinline__ void cross3(const double* p, const double* q, double* o)
{
    o[0] = p[1] * q[2] - p[2] * q[1];
    o[1] = p[2] * q[0] - p[0] * q[2];
    o[2] = p[0] * q[1] - p[1] * q[0];
}

struct LoadArgs {
    const float4* seg_a;
    const float4* seg_b;
    long long m;
    const float* u_ind;  // [3][m]
    double omega[3], hub[3], u_inf[3];
    const float4* rings;  // [n][4]
    const float4* normal;
    const double* gamma;
    const double* gamma_prev;  // or null
    long long n;
    double dt, rho;
    double* terms;  // [m + n][6]
};

__global__ void loads_terms_kernel(const LoadArgs L)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double f[3] = {0, 0, 0}, rel[3] = {0, 0, 0};
    if (i < L.m) {
        const float4 a = L.seg_a[i], b = L.seg_b[i];
        const double A[3] = {a.x, a.y, a.z}, B[3] = {b.x, b.y, b.z};
        double dl[3], w[3], V[3];
        for (int c = 0; c < 3; ++c) {
            rel[c] = 0.5 * (A[c] + B[c]) - L.hub[c];
            dl[c] = B[c] - A[c];
        }
        cross3(L.omega, rel, w);
        for (int c = 0; c < 3; ++c) V[c] = L.u_inf[c] - w[c] + (double)L.u_ind[c * L.m + i];
        cross3(V, dl, f);
        for (int c = 0; c < 3; ++c) f[c] *= L.rho * (double)a.w;
    } else if (i < L.m + L.n) {
        const long long p = i - L.m;
        if (L.gamma_prev) {
            double C[4][3];
            for (int k = 0; k < 4; ++k) {
                const float4 q = L.rings[4 * p + k];
                C[k][0] = q.x, C[k][1] = q.y, C[k][2] = q.z;
            }
            double d1[3], d2[3], cr[3];
            for (int c = 0; c < 3; ++c) {
                d1[c] = C[2][c] - C[0][c];
                d2[c] = C[3][c] - C[1][c];
                rel[c] = 0.25 * (C[0][c] + C[1][c] + C[2][c] + C[3][c]) - L.hub[c];
            }
            cross3(d1, d2, cr);
            const double area = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            const double k = L.rho * (L.gamma[p] - L.gamma_prev[p]) / L.dt * area;
            const float4 nn = L.normal[p];
            f[0] = k * nn.x, f[1] = k * nn.y, f[2] = k * nn.z;
        }
    } else {
        return;
    }
    double mom[3];
    cross3(rel, f, mom);
    double* t = L.terms + 6 * i;
    for (int c = 0; c < 3; ++c) t[c] = f[c], t[3 + c] = mom[c];
}

// out[0..5] = sum of terms[0..count), thread t summing items t, t + T, ... in order,
// then a fixed tree over the threads.
constexpr int LOAD_RED_THREADS = 256;
__global__ void __launch_bounds__(LOAD_RED_THREADS) loads_reduce_kernel(const double* __restrict__ terms,
                                                                        long long count, double* __restrict__ out)
{
    __shared__ double s[6][LOAD_RED_THREADS];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long i = threadIdx.x; i < count; i += LOAD_RED_THREADS)
        for (int c = 0; c < 6; ++c) acc[c] += terms[6 * i + c];
    for (int c = 0; c < 6; ++c) s[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = LOAD_RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 6; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 6) out[threadIdx.x] = s[threadIdx.x][0];
}

// FP32 targets at the midpoints of m segments.
__global__ void segment_midpoints_kernel(const float4* __restrict__ a, const float4* __restrict__ b, long long m,
                                         float4* __restrict__ tgt)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float4 p = a[i], q = b[i];
    tgt[i] = make_float4(0.5f * (p.x + q.x), 0.5f * (p.y + q.y), 0.5f * (p.z + q.z), 0.f);
}

size_t loads_workspace(long long m, long long n) { return ((size_t)(m + n) * 6 * sizeof(double) + 255) & ~size_t(255); }

cudaError_t run_segment_midpoints(const float* seg_a, const float* seg_b, long long m, float* tgt, cudaStream_t st)
{
    if (m == 0) return cudaSuccess;
    trace_launch();
    segment_midpoints_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const float4*>(seg_a), reinterpret_cast<const float4*>(seg_b), m,
        reinterpret_cast<float4*>(tgt));
    return cudaGetLastError();
}

cudaError_t run_blade_loads(const float* seg_a, const float* seg_b, long long m, const float* u_ind,
                            const double* omega, const double* hub, const double* u_inf, const float* rings,
                            const float* normal, const double* gamma, const double* gamma_prev, long long n, double dt,
                            double rho, double* out, char* ws, cudaStream_t st)
{
    LoadArgs L;
    L.seg_a = reinterpret_cast<const float4*>(seg_a);
    L.seg_b = reinterpret_cast<const float4*>(seg_b);
    L.m = m;
    L.u_ind = u_ind;
    for (int c = 0; c < 3; ++c) L.omega[c] = omega[c], L.hub[c] = hub[c], L.u_inf[c] = u_inf[c];
    L.rings = reinterpret_cast<const float4*>(rings);
    L.normal = reinterpret_cast<const float4*>(normal);
    L.gamma = gamma;
    L.gamma_prev = gamma_prev;
    L.n = n;
    L.dt = dt;
    L.rho = rho;
    L.terms = reinterpret_cast<double*>(ws);
    const long long count = m + n;
    if (count > 0) {
        trace_launch();
        loads_terms_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(L);
    }
    trace_launch();
    loads_reduce_kernel<<<1, LOAD_RED_THREADS, 0, st>>>(L.terms, count, out);
    return cudaGetLastError();
}

}  // namespace vpm
