// Blade influence-coefficient (AIC) system of the vortex-lattice method (Sec. II.A):
// the Neumann condition at the collocation points, A Gamma_b = b.
//
//  * aic_build: A[k][l] = u(ring l, unit circulation)(y_k) . n_k, each ring the four
//    Vatistas-cored segments of its corners; b[k] = -(v_rel,k + w_k) . n_k in FP64.
//  * aic_solve: A factored once in FP32 by a blocked right-looking LU with partial
//    pivoting (panel kernel, triangular solve of the block row, FP32 update of the
//    trailing matrix), then iterative refinement: the residual r = b - A x is formed
//    in FP64 from the FP32 matrix, the correction solved with the FP32 factors and
//    added to x in FP64, until the normwise backward error is below tol.
#include <math.h>

#include "vpm_internal.h"

namespace vpm {

// ---------------------------------------------------------------------------
// AIC build.
// ---------------------------------------------------------------------------
// Velocity of a unit-circulation segment p->q at y (FP32), Vatistas exponent vn;
// zero within 1e-10 |q - p| (or 1e-15 m) of an end point or where the regularised denominator
// vanishes.  Without the 1/(4 pi) factor.
__device__ __forceinline__ void seg_u(float4 p, float4 q, float3 y, float core, int vn, float& ux, float& uy,
                                      float& uz)
{
    const float r0x = q.x - p.x, r0y = q.y - p.y, r0z = q.z - p.z;
    const float r1x = y.x - p.x, r1y = y.y - p.y, r1z = y.z - p.z;
    const float r2x = y.x - q.x, r2y = y.y - q.y, r2z = y.z - q.z;
    const float L2 = r0x * r0x + r0y * r0y + r0z * r0z;
    const float n1 = r1x * r1x + r1y * r1y + r1z * r1z;
    const float n2 = r2x * r2x + r2y * r2y + r2z * r2z;
    const float cx = r0y * r1z - r0z * r1y, cy = r0z * r1x - r0x * r1z, cz = r0x * r1y - r0y * r1x;
    const float c2 = cx * cx + cy * cy + cz * cz;
    const float thr = fmaxf(1e-20f * L2, 1e-30f);
    ux = uy = uz = 0.f;
    if (!(n1 > thr && n2 > thr)) return;
    const float cl2 = core * core * L2;
    float D = vn == 2 ? sqrtf(c2 * c2 + cl2 * cl2) : c2 + cl2;
    if (!(D > 0.f)) return;
    const float d = (r0x * r1x + r0y * r1y + r0z * r1z) * rsqrtf(n1) - (r0x * r2x + r0y * r2y + r0z * r2z) * rsqrtf(n2);
    const float s = d / D;
    ux = s * cx;
    uy = s * cy;
    uz = s * cz;
}

__global__ void __launch_bounds__(256) aic_build_kernel(const float4* __restrict__ rings,
                                                        const float4* __restrict__ colloc,
                                                        const float4* __restrict__ normal, int n, float core, int vn,
                                                        const float4* __restrict__ v_rel, const float* __restrict__ w,
                                                        float* __restrict__ A, double* __restrict__ b)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y * blockDim.y + threadIdx.y;
    if (k >= n) return;
    const float4 yk4 = colloc[k], nk = normal[k];
    if (l < n) {
        const float3 yk = make_float3(yk4.x, yk4.y, yk4.z);
        const float4 c0 = rings[4 * l], c1 = rings[4 * l + 1], c2 = rings[4 * l + 2], c3 = rings[4 * l + 3];
        float tx = 0.f, ty = 0.f, tz = 0.f, ux, uy, uz;
        seg_u(c0, c1, yk, core, vn, ux, uy, uz);
        tx += ux, ty += uy, tz += uz;
        seg_u(c1, c2, yk, core, vn, ux, uy, uz);
        tx += ux, ty += uy, tz += uz;
        seg_u(c2, c3, yk, core, vn, ux, uy, uz);
        tx += ux, ty += uy, tz += uz;
        seg_u(c3, c0, yk, core, vn, ux, uy, uz);
        tx += ux, ty += uy, tz += uz;
        A[(size_t)k * n + l] = (tx * nk.x + ty * nk.y + tz * nk.z) * 0.0795774715459476679f;
    }
    if (b && l == 0) {
        const float4 v = v_rel[k];
        double vx = v.x, vy = v.y, vz = v.z;
        if (w) vx += w[k], vy += w[n + k], vz += w[2 * n + k];
        b[k] = -(vx * nk.x + vy * nk.y + vz * nk.z);
    }
}

cudaError_t run_aic_build(const float* rings, const float* colloc, const float* normal, int n, float core, int vn,
                          const float* v_rel, const float* w_ind, float* A, double* b, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8);
    trace_launch();
    aic_build_kernel<<<grd, blk, 0, st>>>(reinterpret_cast<const float4*>(rings),
                                          reinterpret_cast<const float4*>(colloc),
                                          reinterpret_cast<const float4*>(normal), n, core, vn,
                                          reinterpret_cast<const float4*>(v_rel), w_ind, A, b);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 LU with partial pivoting, panel width NB.
// ---------------------------------------------------------------------------
constexpr int NB = 32;
constexpr int LU_THREADS = 1024;

// Factors columns [k0, k0 + nb) of rows [k0, n) in place with partial pivoting (one
// block).  The panel is held in shared memory (rows padded to nb + 1 floats) when it
// fits, else worked on in global memory; only the panel's own columns are swapped
// here, the other columns by lu_laswp_kernel.
template <bool SMEM>
__global__ void __launch_bounds__(LU_THREADS) lu_panel_kernel(float* __restrict__ A, int n, int k0, int nb,
                                                              int* __restrict__ piv, int* __restrict__ info)
{
    extern __shared__ float P[];
    __shared__ float sv[32];
    __shared__ int si[32];
    const int rows = n - k0, ld = SMEM ? nb + 1 : n;
    float* base = SMEM ? P : A + (size_t)k0 * n + k0;
    if (SMEM) {
        for (int e = threadIdx.x; e < rows * nb; e += blockDim.x) {
            const int r = e / nb, c = e % nb;
            P[r * ld + c] = A[(size_t)(k0 + r) * n + k0 + c];
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < nb; ++j) {
        // pivot: per-warp candidates, one barrier, then every warp reduces the candidates itself
        float v = -1.f;
        int idx = 0x7fffffff;
        for (int r = j + threadIdx.x; r < rows; r += blockDim.x) {
            const float a = fabsf(base[(size_t)r * ld + j]);
            if (a > v || (a == v && r < idx)) v = a, idx = r;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (ov > v || (ov == v && oi < idx)) v = ov, idx = oi;
        }
        if (lane == 0) sv[warp] = v, si[warp] = idx;
        __syncthreads();
        v = lane < nw ? sv[lane] : -1.f;
        idx = lane < nw ? si[lane] : 0x7fffffff;
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (ov > v || (ov == v && oi < idx)) v = ov, idx = oi;
        }
        const float best = v;
        const int p = idx;
        if (!(best > 0.f)) {  // exactly singular column (or NaN): keep going, report
            if (threadIdx.x == 0) {
                piv[k0 + j] = k0 + j;
                if (*info == 0) *info = k0 + j + 1;
            }
            __syncthreads();
            continue;
        }
        if (threadIdx.x == 0) piv[k0 + j] = k0 + p;
        if (p != j && threadIdx.x < nb) {
            const int c = threadIdx.x;
            const float t = base[(size_t)j * ld + c];
            base[(size_t)j * ld + c] = base[(size_t)p * ld + c];
            base[(size_t)p * ld + c] = t;
        }
        __syncthreads();  // swapped rows and the reduction slots are settled
        const float inv = 1.0f / base[(size_t)j * ld + j];
        for (int r = j + 1 + threadIdx.x; r < rows; r += blockDim.x) {
            float* row = base + (size_t)r * ld;
            const float l = row[j] * inv;
            row[j] = l;
            for (int c = j + 1; c < nb; ++c) row[c] = fmaf(-l, base[(size_t)j * ld + c], row[c]);
        }
        __syncthreads();
    }
    if (SMEM) {
        for (int e = threadIdx.x; e < rows * nb; e += blockDim.x) {
            const int r = e / nb, c = e % nb;
            A[(size_t)(k0 + r) * n + k0 + c] = P[r * ld + c];
        }
    }
}

// Applies the row exchanges of panel [k0, k0 + nb) to every column outside it.
__global__ void __launch_bounds__(256) lu_laswp_kernel(float* __restrict__ A, int n, int k0, int nb,
                                                       const int* __restrict__ piv)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n - nb) return;
    if (c >= k0) c += nb;
    for (int j = k0; j < k0 + nb; ++j) {
        const int p = piv[j];
        if (p != j) {
            const float t = A[(size_t)j * n + c];
            A[(size_t)j * n + c] = A[(size_t)p * n + c];
            A[(size_t)p * n + c] = t;
        }
    }
}

// U12 = L11^-1 A12 for the block row [k0, k0+nb), columns [k0+nb, n): one thread per column.
__global__ void __launch_bounds__(256) lu_trsm_kernel(float* __restrict__ A, int n, int k0, int nb)
{
    __shared__ float L[NB][NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, p = e % nb;
        L[i][p] = A[(size_t)(k0 + i) * n + k0 + p];
    }
    __syncthreads();
    const int c = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    float x[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        if (i < nb) {
            float s = A[(size_t)(k0 + i) * n + c];
#pragma unroll
            for (int p = 0; p < NB; ++p)
                if (p < i) s -= L[i][p] * x[p];
            x[i] = s;
            A[(size_t)(k0 + i) * n + c] = s;
        }
    }
}

// A22 -= L21 U12 over rows/cols [k0+nb, n): 64x64 output tile per block, 4x4 per thread.
__global__ void __launch_bounds__(256) lu_update_kernel(float* __restrict__ A, int n, int k0, int nb)
{
    __shared__ float Ls[64][NB + 1];
    __shared__ float Us[NB][64 + 1];
    const int s0 = k0 + nb;
    const int r0 = s0 + blockIdx.y * 64, c0 = s0 + blockIdx.x * 64;
    for (int e = threadIdx.x; e < 64 * NB; e += blockDim.x) {
        const int i = e / NB, p = e % NB;
        const int r = r0 + i;
        Ls[i][p] = (r < n && p < nb) ? A[(size_t)r * n + k0 + p] : 0.f;
        const int pp = e / 64, cc = e % 64;
        const int c = c0 + cc;
        Us[pp][cc] = (c < n && pp < nb) ? A[(size_t)(k0 + pp) * n + c] : 0.f;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4] = {};
#pragma unroll 8
    for (int p = 0; p < NB; ++p) {
        float a[4], bb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = Ls[ty * 4 + q][p], bb[q] = Us[p][tx * 4 + q];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[q][w] = fmaf(a[q], bb[w], acc[q][w]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = r0 + ty * 4 + q;
        if (r >= n) continue;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int c = c0 + tx * 4 + w;
            if (c < n) A[(size_t)r * n + c] -= acc[q][w];
        }
    }
}

// Solves (LU) z = P r in FP32 for a FP64 right-hand side, one block, the vector in
// shared memory; z returned in FP64.  Each 32-row diagonal block is solved by one
// warp, then every thread updates one remaining row with a 32-long dot product.
__global__ void __launch_bounds__(LU_THREADS) lu_solve_kernel(const float* __restrict__ LU,
                                                              const int* __restrict__ piv, int n,
                                                              const double* __restrict__ rhs, double* __restrict__ z)
{
    extern __shared__ float y[];  // y[n], then the pivots as int[n]
    int* sp = reinterpret_cast<int*>(y + n);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < n; i += blockDim.x) y[i] = (float)rhs[i], sp[i] = piv[i];
    __syncthreads();
    if (tid == 0)  // the row exchanges in order, on shared memory
        for (int j = 0; j < n; ++j) {
            const int p = sp[j];
            if (p != j) {
                const float t = y[j];
                y[j] = y[p];
                y[p] = t;
            }
        }
    __syncthreads();
    // forward: L (unit lower)
    for (int b0 = 0; b0 < n; b0 += 32) {
        const int bn = min(32, n - b0);
        if (warp == 0) {
            float v = lane < bn ? y[b0 + lane] : 0.f;
            const float* row = LU + (size_t)(b0 + (lane < bn ? lane : 0)) * n + b0;
            float lr[32];
#pragma unroll
            for (int p = 0; p < 32; ++p) lr[p] = p < bn ? row[p] : 0.f;  // all loads in flight at once
#pragma unroll
            for (int p = 0; p < 32; ++p) {
                const float yp = __shfl_sync(0xffffffffu, v, p);
                if (lane > p && lane < bn) v = fmaf(-lr[p], yp, v);
            }
            if (lane < bn) y[b0 + lane] = v;
        }
        __syncthreads();
        for (int i = b0 + bn + tid; i < n; i += blockDim.x) {
            const float* row = LU + (size_t)i * n + b0;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            int p = 0;
            for (; p + 4 <= bn; p += 4) {
                s0 = fmaf(row[p], y[b0 + p], s0);
                s1 = fmaf(row[p + 1], y[b0 + p + 1], s1);
                s2 = fmaf(row[p + 2], y[b0 + p + 2], s2);
                s3 = fmaf(row[p + 3], y[b0 + p + 3], s3);
            }
            for (; p < bn; ++p) s0 = fmaf(row[p], y[b0 + p], s0);
            y[i] -= (s0 + s1) + (s2 + s3);
        }
        __syncthreads();
    }
    // backward: U
    for (int b1 = n; b1 > 0; b1 -= 32) {
        const int b0 = max(0, b1 - 32), bn = b1 - b0;
        if (warp == 0) {
            float v = lane < bn ? y[b0 + lane] : 0.f;
            const float* row = LU + (size_t)(b0 + (lane < bn ? lane : 0)) * n + b0;
            float lr[32];
#pragma unroll
            for (int p = 0; p < 32; ++p) lr[p] = p < bn ? row[p] : 1.f;
#pragma unroll
            for (int p = 31; p >= 0; --p) {
                if (p < bn) {
                    if (lane == p) v /= lr[p];
                    const float yp = __shfl_sync(0xffffffffu, v, p);
                    if (lane < p) v = fmaf(-lr[p], yp, v);
                }
            }
            if (lane < bn) y[b0 + lane] = v;
        }
        __syncthreads();
        for (int i = tid; i < b0; i += blockDim.x) {
            const float* row = LU + (size_t)i * n + b0;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            int p = 0;
            for (; p + 4 <= bn; p += 4) {
                s0 = fmaf(row[p], y[b0 + p], s0);
                s1 = fmaf(row[p + 1], y[b0 + p + 1], s1);
                s2 = fmaf(row[p + 2], y[b0 + p + 2], s2);
                s3 = fmaf(row[p + 3], y[b0 + p + 3], s3);
            }
            for (; p < bn; ++p) s0 = fmaf(row[p], y[b0 + p], s0);
            y[i] -= (s0 + s1) + (s2 + s3);
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += blockDim.x) z[i] = (double)y[i];
}

// r = b - A x in FP64 (A's FP32 entries promoted exactly); also row |A| sums on the first pass.
__global__ void __launch_bounds__(256) residual_kernel(const float* __restrict__ A, const double* __restrict__ b,
                                                       const double* __restrict__ x, int n, double* __restrict__ r,
                                                       double* __restrict__ rowabs)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    double s = 0.0, a = 0.0;
    for (int c = lane; c < n; c += 32) {
        const double v = (double)A[(size_t)i * n + c];
        s = fma(v, x[c], s);
        a += fabs(v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        a += __shfl_xor_sync(0xffffffffu, a, o);
    }
    if (lane == 0) {
        r[i] = b[i] - s;
        if (rowabs) rowabs[i] = a;
    }
}

// out = (max|r|, max|x|, max|b|, max rowabs) ; one block.
__global__ void __launch_bounds__(1024) norms_kernel(const double* __restrict__ r, const double* __restrict__ x,
                                                     const double* __restrict__ b,
                                                     const double* __restrict__ rowabs, int n,
                                                     double* __restrict__ out)
{
    __shared__ double s[4][32];
    double m[4] = {0, 0, 0, 0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        m[0] = fmax(m[0], fabs(r[i]));
        m[1] = fmax(m[1], fabs(x[i]));
        m[2] = fmax(m[2], fabs(b[i]));
        m[3] = fmax(m[3], rowabs[i]);
        if (!isfinite(r[i]) || !isfinite(x[i])) m[0] = INFINITY;
    }
    for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) m[q] = fmax(m[q], __shfl_xor_sync(0xffffffffu, m[q], o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int q = 0; q < 4; ++q) s[q][w] = m[q];
    __syncthreads();
    if (w == 0) {
        for (int q = 0; q < 4; ++q) {
            double v = lane < (int)(blockDim.x >> 5) ? s[q][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) out[q] = v;
        }
    }
}

__global__ void add_kernel(double* __restrict__ x, const double* __restrict__ d, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += d[i];
}

namespace {
struct AicWs {
    size_t lu, piv, info, r, d, rowabs, norms, bytes;
};
AicWs aic_layout(int n)
{
    Carve cv;
    AicWs w;
    w.lu = cv.take((size_t)n * n * sizeof(float));
    w.piv = cv.take((size_t)n * sizeof(int));
    w.info = cv.take(sizeof(int));
    w.r = cv.take((size_t)n * sizeof(double));
    w.d = cv.take((size_t)n * sizeof(double));
    w.rowabs = cv.take((size_t)n * sizeof(double));
    w.norms = cv.take(4 * sizeof(double));
    w.bytes = cv.off;
    return w;
}
}  // namespace

size_t aic_workspace(int n) { return aic_layout(n).bytes; }

vpm_status run_aic_solve(const float* A, const double* b, double* x, int n, double tol, int max_iter, int* iters,
                         double* berr, char* ws, cudaStream_t st, const char** msg)
{
    if (iters) *iters = 0;
    if (berr) *berr = 0.0;
    if (n == 0) return VPM_OK;
    const AicWs L = aic_layout(n);
    float* LU = reinterpret_cast<float*>(ws + L.lu);
    int* piv = reinterpret_cast<int*>(ws + L.piv);
    int* info = reinterpret_cast<int*>(ws + L.info);
    double* r = reinterpret_cast<double*>(ws + L.r);
    double* d = reinterpret_cast<double*>(ws + L.d);
    double* rowabs = reinterpret_cast<double*>(ws + L.rowabs);
    double* norms = reinterpret_cast<double*>(ws + L.norms);
#define VPM_CU(call)                                 \
    do {                                             \
        if ((call) != cudaSuccess) {                 \
            *msg = cudaGetErrorString(cudaGetLastError()); \
            return VPM_ERR_CUDA;                     \
        }                                            \
    } while (0)
    VPM_CU(cudaMemcpyAsync(LU, A, (size_t)n * n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    VPM_CU(cudaMemsetAsync(info, 0, sizeof(int), st));
    // panel width 32 when the panel fits in shared memory, else 16, else a global-memory panel
    const int maxsm = 200 * 1024;
    const int pnb = ((size_t)n * 33 * sizeof(float) <= (size_t)maxsm) ? 32 : 16;
    const bool psmem = (size_t)n * (pnb + 1) * sizeof(float) <= (size_t)maxsm;
    if (psmem) {
        VPM_CU(cudaFuncSetAttribute(lu_panel_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    }
    VPM_CU(cudaFuncSetAttribute(lu_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(n * (sizeof(float) + sizeof(int)))));
    for (int k0 = 0; k0 < n; k0 += pnb) {
        const int nb = n - k0 < pnb ? n - k0 : pnb;
        trace_launch();
        if (psmem)
            lu_panel_kernel<true><<<1, LU_THREADS, (size_t)(n - k0) * (nb + 1) * sizeof(float), st>>>(LU, n, k0, nb,
                                                                                                     piv, info);
        else
            lu_panel_kernel<false><<<1, LU_THREADS, 0, st>>>(LU, n, k0, nb, piv, info);
        if (n - nb > 0) {
            trace_launch();
            lu_laswp_kernel<<<(n - nb + 255) / 256, 256, 0, st>>>(LU, n, k0, nb, piv);
        }
        const int rest = n - k0 - nb;
        if (rest > 0) {
            trace_launch();
            lu_trsm_kernel<<<(rest + 255) / 256, 256, 0, st>>>(LU, n, k0, nb);
            dim3 g((rest + 63) / 64, (rest + 63) / 64);
            trace_launch();
            lu_update_kernel<<<g, 256, 0, st>>>(LU, n, k0, nb);
        }
    }
    VPM_CU(cudaGetLastError());
    int hinfo = 0;
    VPM_CU(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    VPM_CU(cudaStreamSynchronize(st));
    if (hinfo != 0) {
        *msg = "aic_solve: matrix is singular in FP32 (zero pivot)";
        return VPM_ERR_NOT_CONVERGED;
    }
    trace_launch();
    lu_solve_kernel<<<1, LU_THREADS, n * (sizeof(float) + sizeof(int)), st>>>(LU, piv, n, b, x);
    double h[4];
    double best = INFINITY;
    for (int it = 0;; ++it) {
        trace_launch();
        residual_kernel<<<(n * 32 + 255) / 256, 256, 0, st>>>(A, b, x, n, r, it == 0 ? rowabs : nullptr);
        trace_launch();
        norms_kernel<<<1, 1024, 0, st>>>(r, x, b, rowabs, n, norms);
        VPM_CU(cudaGetLastError());
        VPM_CU(cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, st));
        VPM_CU(cudaStreamSynchronize(st));
        const double den = h[3] * h[1] + h[2];
        const double be = den > 0.0 ? h[0] / den : (h[0] > 0.0 ? INFINITY : 0.0);
        best = be < best ? be : best;
        if (iters) *iters = it;
        if (berr) *berr = be;
        if (be <= tol) return VPM_OK;
        if (it >= max_iter || !isfinite(be)) {
            *msg = "aic_solve: backward error above tol after max_iter refinement steps";
            return VPM_ERR_NOT_CONVERGED;
        }
        trace_launch();
        lu_solve_kernel<<<1, LU_THREADS, n * (sizeof(float) + sizeof(int)), st>>>(LU, piv, n, r, d);
        trace_launch();
        add_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, d, n);
    }
#undef VPM_CU
}

}  // namespace vpm
