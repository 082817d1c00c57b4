// Blade influence-coefficient (AIC) system of the vortex-lattice method (Sec. II.A):
// the Neumann condition at the collocation points, A Gamma_b = b.
//
//  * aic_build: A[k][l] = u(ring l, unit circulation)(y_k) . n_k, each ring the four
//    Vatistas-cored segments of its corners; b[k] = -(v_rel,k + w_k) . n_k in FP64.
//  * aic_solve: A factored once in FP32 by a blocked right-looking LU with partial
//    pivoting (panel kernel with one block barrier per column, row exchanges and the
//    block row U12 in one kernel, FP32 update of the trailing matrix), then iterative
//    refinement: the residual r = b - A x is formed in FP64 from the FP32 matrix, the
//    correction solved with the FP32 factors (read through a transposed copy so that
//    the substitutions load coalesced columns) and added to x in FP64, until the
//    normwise backward error is below tol.
#include <math.h>

#include <algorithm>

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
//
// Per panel [k0, k0 + nb): lu_panel_kernel factors the panel's columns (one block),
// lu_rows_kernel applies the panel's row exchanges to every other column and forms
// the block row U12 = L11^-1 A12, lu_update_kernel updates A22 -= L21 U12.  The
// result is LAPACK's: P A = L U with the row exchanges applied to whole rows.
// ---------------------------------------------------------------------------
constexpr int NB = 32;
constexpr int LU_THREADS = 1024;  // the triangular solves

// The end of a panel, after a barrier that made the final position map `pos2phys`
// visible (and with *nmov zeroed before it): lists the changed positions as (source,
// destination) moves -- at most 2 nb, the panel's own rows and the rows they displaced
// -- and applies them to the permutation.
template <int NT>
__device__ __forceinline__ void panel_moves(const int* pos2phys, int rows, int k0, int* __restrict__ perm,
                                            int* __restrict__ moves, int* nmov)
{
    const int tid = threadIdx.x;
    for (int i = tid; i < rows; i += NT) {
        const int s = pos2phys[i];
        if (s != i) {
            const int m = atomicAdd(nmov, 1);
            moves[1 + 2 * m] = s;
            moves[2 + 2 * m] = i;
        }
    }
    __syncthreads();
    const int cnt = *nmov;
    int pv = 0;
    if (tid < cnt) pv = perm[k0 + moves[1 + 2 * tid]];
    __syncthreads();  // every move's source is read before any destination is written
    if (tid < cnt) perm[k0 + moves[2 + 2 * tid]] = pv;
    if (tid == 0) moves[0] = cnt;
}

// Factors columns [k0, k0 + nb) of rows [k0, n) with partial pivoting (one block of
// PANEL_THREADS).  The panel is copied into rows of PLD floats (16-byte aligned, so a
// row is updated with float4 accesses), the first `srows` of them in shared memory and
// the rest in the global scratch `pscratch`.  Rows never move while the panel is
// worked on: thread t owns physical rows t, t + PANEL_THREADS, ..., and the row
// exchanges are kept as a logical-position <-> physical-row map (thread 0 only), so
// that a column costs one block barrier:
//   1. each thread measures column j on its live rows; a 32-bit key orders |a| and
//      puts NaN below every number (0 = no live row); the warp takes the maximum with
//      redux.sync, the lowest lane holding it wins, and the warp publishes that row's
//      copy, key and index in a slot of a two-deep ring;
//   2. one barrier; every warp reduces the published keys the same way, so all
//      threads know the pivot row and read it from the winning slot;
//   3. every thread eliminates column j from its live rows.
// The ring is two deep because slot j & 1 is rewritten only at column j + 2, after the
// barrier of column j + 1, by which time every thread has finished using it.  At the
// end the rows are written back in their logical order, the positions that changed
// are listed as (source, destination) moves for lu_rows_kernel, and the permutation
// `perm` (original row index of each position) is updated with the same moves.
// A column whose largest candidate is not positive (all zero or NaN) sets *info to
// its 1-based index (first such column) and is not eliminated.
constexpr int PANEL_THREADS = 512;
constexpr int PANEL_WARPS = PANEL_THREADS / 32;
constexpr int PLD = NB + 4;
static_assert(VPM_MAX_AIC <= 32 * PANEL_THREADS, "row ownership mask is 32 bits");

template <bool ALL_SMEM>
__global__ void __launch_bounds__(PANEL_THREADS, 1) lu_panel_kernel(float* __restrict__ A, int n, int k0, int nb,
                                                                 int* __restrict__ info, int* __restrict__ perm,
                                                                 int* __restrict__ moves, float* pscratch, int srows)
{
    constexpr int NT = PANEL_THREADS;
    extern __shared__ __align__(16) float psm[];  // srows * PLD floats, then pos2phys[rows], phys2pos[rows]
    __shared__ __align__(16) float crow[2][PANEL_WARPS][NB];
    __shared__ unsigned ckey[2][PANEL_WARPS];
    __shared__ int cidx[2][PANEL_WARPS];
    __shared__ float cpiv[2][PANEL_WARPS];
    __shared__ int nmov;
    const int rows = n - k0;
    int* pos2phys = reinterpret_cast<int*>(psm + (size_t)srows * PLD);
    int* phys2pos = pos2phys + rows;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // Calls f with row r of the panel copy.  The two branches give the compiler a
    // shared-memory and a global pointer, so each access is a plain shared or global
    // one (ALL_SMEM: every row is in shared memory).
    auto with_row = [&](int r, auto&& f) {
        if (ALL_SMEM || r < srows) return f(psm + (size_t)r * PLD);
        return f(pscratch + (size_t)(r - srows) * PLD);
    };
    if (k0 == 0) {
        for (int i = tid; i < n; i += NT) perm[i] = i;
        if (tid == 0) *info = 0;
    }
    const int nmine = tid < rows ? (rows - 1 - tid) / NT + 1 : 0;
    for (int t = 0; t < nmine; ++t) {  // my rows: 32 independent loads each, then float4 stores
        const int r = tid + t * NT;
        const float* src = A + (size_t)(k0 + r) * n + k0;
        float v[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) v[c] = c < nb ? src[c] : 0.f;  // a narrow last panel is zero-filled
        with_row(r, [&](float* row) {
#pragma unroll
            for (int c4 = 0; c4 < NB / 4; ++c4)
                reinterpret_cast<float4*>(row)[c4] = make_float4(v[4 * c4], v[4 * c4 + 1], v[4 * c4 + 2], v[4 * c4 + 3]);
        });
    }
    for (int i = tid; i < rows; i += NT) pos2phys[i] = i, phys2pos[i] = i;
    if (tid == 0) nmov = 0;
    __syncthreads();

    unsigned done = 0;  // bit t: my row tid + t * NT is a pivot row already
    for (int j = 0; j < nb; ++j) {
        unsigned key = 0;
        int rb = 0;
        for (int t = 0; t < nmine; ++t) {
            if (done >> t & 1u) continue;
            const int r = tid + t * NT;
            const float v = with_row(r, [&](float* row) { return fabsf(row[j]); });
            const unsigned k = v == v ? __float_as_uint(v) + 2u : 1u;
            if (k > key) key = k, rb = r;
        }
        const unsigned wmax = __reduce_max_sync(0xffffffffu, key);
        const int wl = __ffs(__ballot_sync(0xffffffffu, key == wmax)) - 1;
        const int wr = __shfl_sync(0xffffffffu, rb, wl);
        __syncwarp();  // the lanes' row updates are visible to the whole warp
        // the candidate row with its columns <= j zeroed (those keep their values in the
        // elimination), and its entry in column j
        if (lane < NB / 4)
            with_row(wr, [&](float* row) {
                float4 v = reinterpret_cast<const float4*>(row)[lane];
                const int c = 4 * lane;
                if (c <= j) v.x = 0.f;
                if (c + 1 <= j) v.y = 0.f;
                if (c + 2 <= j) v.z = 0.f;
                if (c + 3 <= j) v.w = 0.f;
                reinterpret_cast<float4*>(crow[j & 1][warp])[lane] = v;
                if (lane == (j >> 2)) cpiv[j & 1][warp] = row[j];
            });
        if (lane == 0) ckey[j & 1][warp] = wmax, cidx[j & 1][warp] = wr;
        __syncthreads();
        const unsigned k2 = lane < PANEL_WARPS ? ckey[j & 1][lane] : 0u;
        const unsigned bmax = __reduce_max_sync(0xffffffffu, k2);
        const int ws = __ffs(__ballot_sync(0xffffffffu, lane < PANEL_WARPS && k2 == bmax)) - 1;
        const int q = cidx[j & 1][ws];
        const bool ok = bmax > 2u;  // the column's largest |a| is a positive number
        if ((q & (NT - 1)) == tid) done |= 1u << (q / NT);
        if (tid == 0) {
            const int pos = phys2pos[q], x = pos2phys[j];
            pos2phys[j] = q, pos2phys[pos] = x;
            phys2pos[q] = j, phys2pos[x] = pos;
            if (!ok && *info == 0) *info = k0 + j + 1;
        }
        if (ok) {
            const float4* u4 = reinterpret_cast<const float4*>(crow[j & 1][ws]);
            const int c4s = j >> 2;
            float4 uu[NB / 4];
#pragma unroll
            for (int c4 = 0; c4 < NB / 4; ++c4) uu[c4] = u4[c4];
            const float rp = __frcp_rn(cpiv[j & 1][ws]);
            for (int t = 0; t < nmine; ++t) {
                if (done >> t & 1u) continue;
                with_row(tid + t * NT, [&](float* row) {
                    const float l = row[j] * rp;
                    row[j] = l;
                    const float ml = -l;
#pragma unroll
                    for (int c4 = 0; c4 < NB / 4; ++c4) {
                        if (c4 < c4s) continue;  // the same for every thread
                        float4 a = reinterpret_cast<float4*>(row)[c4];
                        a.x = fmaf(ml, uu[c4].x, a.x);
                        a.y = fmaf(ml, uu[c4].y, a.y);
                        a.z = fmaf(ml, uu[c4].z, a.z);
                        a.w = fmaf(ml, uu[c4].w, a.w);
                        reinterpret_cast<float4*>(row)[c4] = a;
                    }
                });
            }
        }
    }
    __syncthreads();  // the position map is final and every row is eliminated
    for (int t = 0; t < nmine; ++t) {  // my rows, to their logical positions
        const int r = tid + t * NT;
        float* dst = A + (size_t)(k0 + phys2pos[r]) * n + k0;
        with_row(r, [&](float* row) {
#pragma unroll
            for (int c4 = 0; c4 < NB / 4; ++c4) {
                const float4 v = reinterpret_cast<const float4*>(row)[c4];
                if (4 * c4 < nb) dst[4 * c4] = v.x;
                if (4 * c4 + 1 < nb) dst[4 * c4 + 1] = v.y;
                if (4 * c4 + 2 < nb) dst[4 * c4 + 2] = v.z;
                if (4 * c4 + 3 < nb) dst[4 * c4 + 3] = v.w;
            }
        });
    }
    panel_moves<NT>(pos2phys, rows, k0, perm, moves, &nmov);
}

// The same factorisation for panels of at most R * NT rows with every row in
// registers.  Thread t owns physical rows t + i * NT (i < R) as 32 registers each,
// rotated so that register c holds column j + c while column j is worked on: the
// elimination of column j writes register c from register c + 1,
//   a[c] = a[c + 1] - l * u[c + 1],
// so every register index is a compile-time constant while the column loop is an
// ordinary loop (a small body that stays in the instruction cache).  The multiplier
// l of each row goes to the shared-memory buffer Lb[row][column]; the pivot row's
// remaining entries (its U row) to Ub[j][column].  Pivot search, publication and the
// one barrier per column are those of lu_panel_kernel.  The panel is read and written
// back with coalesced row accesses staged through Lb.
template <int R, int NT>
__global__ void __launch_bounds__(NT, 1) lu_panel_reg_kernel(float* __restrict__ A, int n, int k0, int nb,
                                                             int* __restrict__ info, int* __restrict__ perm,
                                                             int* __restrict__ moves)
{
    constexpr int NW = NT / 32;
    constexpr int LDL = NB + 1;
    static_assert(NW <= 32, "one warp reduces the published candidates");
    static_assert(R <= 6, "the publication switch covers six rows per thread");
    extern __shared__ float Lb[];  // [rows][LDL], then pos2phys[rows], phys2pos[rows]
    __shared__ __align__(16) float crow[2][NW][NB];
    __shared__ float Ub[NB][NB + 1];
    __shared__ unsigned ckey[2][NW];
    __shared__ int cidx[2][NW];
    __shared__ int nmov;
    const int rows = n - k0;
    int* pos2phys = reinterpret_cast<int*>(Lb + (size_t)rows * LDL);
    int* phys2pos = pos2phys + rows;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (k0 == 0) {
        for (int i = tid; i < n; i += NT) perm[i] = i;
        if (tid == 0) *info = 0;
    }
    // stage the panel in Lb: a warp per row, a lane per column, every copy in flight at
    // once (cp.async, one wait); a narrow last panel is zero-filled
    for (int r = warp; r < rows; r += NW) {
        float* dst = Lb + (size_t)r * LDL + lane;
        if (lane < nb)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)),
                         "l"(A + (size_t)(k0 + r) * n + k0 + lane)
                         : "memory");
        else
            *dst = 0.f;
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    for (int i = tid; i < rows; i += NT) pos2phys[i] = i, phys2pos[i] = i;
    if (tid == 0) nmov = 0;
    __syncthreads();
    float a[R][NB];
    unsigned live = 0;  // bit i: my row tid + i * NT exists and is not a pivot row yet
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = tid + i * NT;
        if (r < rows) live |= 1u << i;
#pragma unroll
        for (int c = 0; c < NB; ++c) a[i][c] = r < rows ? Lb[(size_t)r * LDL + c] : 0.f;
    }
    // (each thread only ever writes Lb rows it owns, which it has just read)
    for (int j = 0; j < nb; ++j) {
        unsigned key = 0;
        int ib = 0;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (live >> i & 1u) {
                const float v = fabsf(a[i][0]);
                const unsigned k = v == v ? __float_as_uint(v) + 2u : 1u;
                if (k > key) key = k, ib = i;
            }
        }
        const unsigned wmax = __reduce_max_sync(0xffffffffu, key);
        const int wl = __ffs(__ballot_sync(0xffffffffu, key == wmax)) - 1;
        if (lane == wl) {
            float4* dst = reinterpret_cast<float4*>(crow[j & 1][warp]);
            auto put = [&](const float* row) {
#pragma unroll
                for (int c4 = 0; c4 < NB / 4; ++c4)
                    dst[c4] = make_float4(row[4 * c4], row[4 * c4 + 1], row[4 * c4 + 2], row[4 * c4 + 3]);
            };
            switch (ib) {  // one branch taken: only the winning row's stores are issued
            case 0: put(a[0]); break;
            case 1: if constexpr (R > 1) put(a[R > 1 ? 1 : 0]); break;
            case 2: if constexpr (R > 2) put(a[R > 2 ? 2 : 0]); break;
            case 3: if constexpr (R > 3) put(a[R > 3 ? 3 : 0]); break;
            case 4: if constexpr (R > 4) put(a[R > 4 ? 4 : 0]); break;
            case 5: if constexpr (R > 5) put(a[R > 5 ? 5 : 0]); break;
            default: break;
            }
            ckey[j & 1][warp] = wmax;
            cidx[j & 1][warp] = tid + ib * NT;
        }
        __syncthreads();
        const unsigned k2 = lane < NW ? ckey[j & 1][lane] : 0u;
        const unsigned bmax = __reduce_max_sync(0xffffffffu, k2);
        const int ws = __ffs(__ballot_sync(0xffffffffu, lane < NW && k2 == bmax)) - 1;
        const int q = cidx[j & 1][ws];
        const bool ok = bmax > 2u;  // the column's largest |a| is a positive number
        const float* u = crow[j & 1][ws];
        if ((q % NT) == tid) live &= ~(1u << (q / NT));
        if (tid == 0) {
            const int pos = phys2pos[q], x = pos2phys[j];
            pos2phys[j] = q, pos2phys[pos] = x;
            phys2pos[q] = j, phys2pos[x] = pos;
            if (!ok && *info == 0) *info = k0 + j + 1;
        }
        if (warp == (j % NW) && j + lane < nb) Ub[j][j + lane] = u[lane];
        const float rp = ok ? __frcp_rn(u[0]) : 0.f;
        float ml[R];  // minus the multipliers; zero for rows that are not live
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const bool lv = live >> i & 1u;
            const float l = ok ? a[i][0] * rp : a[i][0];
            if (lv) Lb[(size_t)(tid + i * NT) * LDL + j] = l;
            ml[i] = (lv && ok) ? -l : 0.f;
        }
        // a[c] = a[c + 1] - l u[c + 1], with u read four entries at a time; registers at or
        // beyond nb - j - 1 hold no column of the panel after this step and are skipped
        float4 u0 = reinterpret_cast<const float4*>(u)[0];
#pragma unroll
        for (int c4 = 0; c4 < NB / 4; ++c4) {
            if (4 * c4 >= nb - 1 - j) break;  // the same for every thread
            const float4 u1 = c4 + 1 < NB / 4 ? reinterpret_cast<const float4*>(u)[c4 + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float un[4] = {u0.y, u0.z, u0.w, u1.x};
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = 4 * c4 + e;
                    a[i][c] = c + 1 < NB ? fmaf(ml[i], un[e], a[i][c + 1]) : 0.f;
                }
            u0 = u1;
        }
    }
    __syncthreads();  // Lb, Ub and the position map are final
    // logical row i: its multipliers from Lb, and for i < nb its U row from Ub
    for (int i = warp; i < rows; i += NW) {
        const int ph = pos2phys[i];
        const float v = (i < nb && lane >= i) ? Ub[i][lane] : Lb[(size_t)ph * LDL + lane];
        if (lane < nb) A[(size_t)(k0 + i) * n + k0 + lane] = v;
    }
    panel_moves<NT>(pos2phys, rows, k0, perm, moves, &nmov);
}

// For every column c outside the panel: moves the panel's exchanged rows
// (A[k0 + dst][c] = old A[k0 + src][c], all sources read first); for c right of the
// panel also solves L11 x = A12[:, c] (unit lower, forward substitution) in place.
constexpr int ROWS_THREADS = 128;
__global__ void __launch_bounds__(ROWS_THREADS, 4) lu_rows_kernel(float* __restrict__ A, int n, int k0, int nb,
                                                               const int* __restrict__ moves)
{
    __shared__ int src[2 * NB], dst[2 * NB];
    __shared__ float L[NB][NB + 1];
    const int cnt = moves[0];
    for (int m = threadIdx.x; m < cnt; m += ROWS_THREADS) src[m] = moves[1 + 2 * m], dst[m] = moves[2 + 2 * m];
    for (int e = threadIdx.x; e < NB * NB; e += ROWS_THREADS) {
        const int i = e / NB, p = e - i * NB;
        L[i][p] = (i < nb && p < nb) ? A[(size_t)(k0 + i) * n + k0 + p] : 0.f;
    }
    __syncthreads();
    int c = blockIdx.x * ROWS_THREADS + threadIdx.x;
    if (c >= n - nb) return;
    if (c >= k0) c += nb;
    float v[2 * NB];
#pragma unroll
    for (int m = 0; m < 2 * NB; ++m)
        if (m < cnt) v[m] = A[(size_t)(k0 + src[m]) * n + c];
#pragma unroll
    for (int m = 0; m < 2 * NB; ++m)
        if (m < cnt) A[(size_t)(k0 + dst[m]) * n + c] = v[m];
    if (c < k0) return;  // a column of L: exchanges only
    float x[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) x[i] = i < nb ? A[(size_t)(k0 + i) * n + c] : 0.f;
#pragma unroll
    for (int p = 0; p < NB - 1; ++p) {  // column-oriented: x[i] -= L[i][p] x[p] for i > p
#pragma unroll
        for (int i = p + 1; i < NB; ++i) x[i] = fmaf(-L[i][p], x[p], x[i]);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i)
        if (i < nb) A[(size_t)(k0 + i) * n + c] = x[i];
}

// A22 -= L21 U12 over rows [k0+nb, n) and columns [cb, ce): 64x64 output tile per
// block, 4x4 per thread.
__global__ void __launch_bounds__(256) lu_update_kernel(float* __restrict__ A, int n, int k0, int nb, int cb, int ce)
{
    __shared__ float Ls[64][NB + 1];
    __shared__ float Us[NB][64 + 1];
    const int s0 = k0 + nb;
    const int r0 = s0 + blockIdx.y * 64, c0 = cb + blockIdx.x * 64;
    for (int e = threadIdx.x; e < 64 * NB; e += blockDim.x) {
        const int i = e / NB, p = e % NB;
        const int r = r0 + i;
        Ls[i][p] = (r < n && p < nb) ? A[(size_t)r * n + k0 + p] : 0.f;
        const int pp = e / 64, cc = e % 64;
        const int c = c0 + cc;
        Us[pp][cc] = (c < ce && pp < nb) ? A[(size_t)(k0 + pp) * n + c] : 0.f;
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
            if (c < ce) A[(size_t)r * n + c] -= acc[q][w];
        }
    }
}

// T = LU^T (32x32 tiles through shared memory), so that the solves read the factors
// column by column with coalesced loads.
__global__ void __launch_bounds__(256) lu_transpose_kernel(const float* __restrict__ LU, float* __restrict__ T,
                                                           int n)
{
    __shared__ float t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = by + k, c = bx + threadIdx.x;
        if (r < n && c < n) t[k][threadIdx.x] = LU[(size_t)r * n + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = bx + k, c = by + threadIdx.x;  // T[r][c] = LU[c][r]
        if (r < n && c < n) T[(size_t)r * n + c] = t[threadIdx.x][k];
    }
}

// Solves (LU) z = P r in FP32 for a FP64 right-hand side (one block, the vector in
// shared memory) and writes z, or adds it to `out` when `accumulate` is set; both in
// FP64.  T = LU^T, so column p of the factors is the contiguous row p of T.  The
// substitution runs over 32-row diagonal blocks: warp 0 solves the block (lane = row,
// a shuffle per column), then every thread updates one remaining row with a 32-long
// dot product.  Nothing the loads of a step fetch depends on the solution, so each
// thread issues its first row's 32 factor entries (coalesced across the warp) and one
// entry of the next diagonal block before the block is solved; the diagonal blocks
// are staged in shared memory one step ahead.
__device__ __forceinline__ float solve_dot(const float* col, int n, const float* yb, int bn)
{
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int p = 0;
    for (; p + 4 <= bn; p += 4) {
        s0 = fmaf(col[(size_t)p * n], yb[p], s0);
        s1 = fmaf(col[(size_t)(p + 1) * n], yb[p + 1], s1);
        s2 = fmaf(col[(size_t)(p + 2) * n], yb[p + 2], s2);
        s3 = fmaf(col[(size_t)(p + 3) * n], yb[p + 3], s3);
    }
    for (; p < bn; ++p) s0 = fmaf(col[(size_t)p * n], yb[p], s0);
    return (s0 + s1) + (s2 + s3);
}

// sum_p t[p] yb[p] over a 32-entry block of the solution (16-byte aligned, read as float4).
__device__ __forceinline__ float dot32(const float* t, const float* yb)
{
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int p4 = 0; p4 < 8; ++p4) {
        const float4 v = reinterpret_cast<const float4*>(yb)[p4];
        s0 = fmaf(t[4 * p4], v.x, s0);
        s1 = fmaf(t[4 * p4 + 1], v.y, s1);
        s0 = fmaf(t[4 * p4 + 2], v.z, s0);
        s1 = fmaf(t[4 * p4 + 3], v.w, s1);
    }
    return s0 + s1;
}

// Element (tid / 32, tid % 32) of the diagonal block starting at c0 (zero outside it).
__device__ __forceinline__ float diag_entry(const float* __restrict__ T, int n, int c0)
{
    const int p = threadIdx.x >> 5, r = threadIdx.x & 31, cn = min(32, n - c0);
    return (c0 >= 0 && c0 < n && p < cn && r < cn) ? T[(size_t)(c0 + p) * n + c0 + r] : 0.f;
}

__global__ void __launch_bounds__(LU_THREADS) lu_solve_kernel(const float* __restrict__ T,
                                                              const int* __restrict__ perm, int n,
                                                              const double* __restrict__ rhs,
                                                              double* __restrict__ out, int accumulate)
{
    extern __shared__ __align__(16) float y[];  // n entries and 32 zeros: a partial block reads zeros past n
    __shared__ float dblk[2][32][33];  // [slot][column p][row r] of a diagonal block
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nblk = (n + 31) / 32;
    for (int i = tid; i < n + 32; i += LU_THREADS) y[i] = i < n ? (float)rhs[perm[i]] : 0.f;
    dblk[0][tid >> 5][tid & 31] = diag_entry(T, n, 0);
    __syncthreads();
    // forward: L (unit lower), blocks in increasing order
    for (int k = 0; k < nblk; ++k) {
        const int b0 = 32 * k, bn = min(32, n - b0), i0 = b0 + bn + tid;
        float t0[32];
#pragma unroll
        for (int p = 0; p < 32; ++p) t0[p] = (i0 < n && p < bn) ? T[(size_t)(b0 + p) * n + i0] : 0.f;
        const float dn = diag_entry(T, n, k + 1 < nblk ? b0 + 32 : -1);
        if (warp == 0) {
            const float(*D)[33] = dblk[k & 1];
            float v = lane < bn ? y[b0 + lane] : 0.f;
#pragma unroll
            for (int p = 0; p < 32; ++p) {
                const float yp = __shfl_sync(0xffffffffu, v, p);
                if (lane > p) v = fmaf(-D[p][lane], yp, v);
            }
            if (lane < bn) y[b0 + lane] = v;
        }
        dblk[(k + 1) & 1][tid >> 5][tid & 31] = dn;
        __syncthreads();
        if (i0 < n) y[i0] -= dot32(t0, y + b0);
        for (int i = i0 + LU_THREADS; i < n; i += LU_THREADS) y[i] -= solve_dot(T + (size_t)b0 * n + i, n, y + b0, bn);
        __syncthreads();
    }
    // backward: U, blocks in decreasing order
    dblk[0][tid >> 5][tid & 31] = diag_entry(T, n, 32 * (nblk - 1));
    __syncthreads();
    for (int k = nblk - 1, s = 0; k >= 0; --k, ++s) {
        const int b0 = 32 * k, bn = min(32, n - b0), i0 = tid;
        float t0[32];
#pragma unroll
        for (int p = 0; p < 32; ++p) t0[p] = (i0 < b0 && p < bn) ? T[(size_t)(b0 + p) * n + i0] : 0.f;
        const float dn = diag_entry(T, n, k > 0 ? b0 - 32 : -1);
        if (warp == 0) {
            const float(*D)[33] = dblk[s & 1];
            float v = lane < bn ? y[b0 + lane] : 0.f;
            const float rd = lane < bn ? 1.0f / D[lane][lane] : 0.f;
#pragma unroll
            for (int p = 31; p >= 0; --p) {
                if (p < bn) {
                    if (lane == p) v *= rd;
                    const float yp = __shfl_sync(0xffffffffu, v, p);
                    if (lane < p) v = fmaf(-D[p][lane], yp, v);
                }
            }
            if (lane < bn) y[b0 + lane] = v;
        }
        dblk[(s + 1) & 1][tid >> 5][tid & 31] = dn;
        __syncthreads();
        if (i0 < b0) y[i0] -= dot32(t0, y + b0);
        for (int i = i0 + LU_THREADS; i < b0; i += LU_THREADS) y[i] -= solve_dot(T + (size_t)b0 * n + i, n, y + b0, bn);
        __syncthreads();
    }
    for (int i = tid; i < n; i += LU_THREADS) out[i] = accumulate ? out[i] + (double)y[i] : (double)y[i];
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


namespace {
struct AicWs {
    size_t lu, t, perm, moves, info, pscratch, r, xbest, rowabs, norms, bytes;
};
AicWs aic_layout(int n)
{
    Carve cv;
    AicWs w;
    w.lu = cv.take((size_t)n * n * sizeof(float));
    w.t = cv.take((size_t)n * n * sizeof(float));
    w.perm = cv.take((size_t)n * sizeof(int));
    w.moves = cv.take((1 + 4 * NB) * sizeof(int));
    w.info = cv.take(sizeof(int));
    w.pscratch = cv.take((size_t)n * PLD * sizeof(float));
    w.r = cv.take((size_t)n * sizeof(double));
    w.xbest = cv.take((size_t)n * sizeof(double));
    w.rowabs = cv.take((size_t)n * sizeof(double));
    w.norms = cv.take(4 * sizeof(double));
    w.bytes = cv.off;
    return w;
}

// Dynamic shared memory of the panel kernel: the two position maps and as many
// panel rows as fit; the remaining rows go to the global scratch.  Panels of at most
// PANEL_REG_ROWS rows use the register kernel (up to PANEL_REG_MAXR rows per thread),
// whose dynamic shared memory is the multiplier buffer and the position maps.
constexpr size_t PANEL_SMEM_MAX = 200 * 1024;
constexpr int PANEL_REG_NT = 256;
constexpr int PANEL_REG_MAXR = 6;
constexpr int PANEL_REG_ROWS = PANEL_REG_MAXR * PANEL_REG_NT;
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
    float* T = reinterpret_cast<float*>(ws + L.t);
    int* perm = reinterpret_cast<int*>(ws + L.perm);
    int* moves = reinterpret_cast<int*>(ws + L.moves);
    int* info = reinterpret_cast<int*>(ws + L.info);
    float* pscratch = reinterpret_cast<float*>(ws + L.pscratch);
    double* r = reinterpret_cast<double*>(ws + L.r);
    double* xbest = reinterpret_cast<double*>(ws + L.xbest);
    double* rowabs = reinterpret_cast<double*>(ws + L.rowabs);
    double* norms = reinterpret_cast<double*>(ws + L.norms);
#define VPM_CU(call)                                       \
    do {                                                   \
        if ((call) != cudaSuccess) {                       \
            *msg = cudaGetErrorString(cudaGetLastError()); \
            return VPM_ERR_CUDA;                           \
        }                                                  \
    } while (0)
    VPM_CU(cudaMemcpyAsync(LU, A, (size_t)n * n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    VPM_CU(cudaFuncSetAttribute(lu_panel_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PANEL_SMEM_MAX));
    VPM_CU(cudaFuncSetAttribute(lu_panel_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PANEL_SMEM_MAX));
    {
        const void* reg_kernels[PANEL_REG_MAXR] = {
            (const void*)lu_panel_reg_kernel<1, PANEL_REG_NT>, (const void*)lu_panel_reg_kernel<2, PANEL_REG_NT>,
            (const void*)lu_panel_reg_kernel<3, PANEL_REG_NT>, (const void*)lu_panel_reg_kernel<4, PANEL_REG_NT>,
            (const void*)lu_panel_reg_kernel<5, PANEL_REG_NT>, (const void*)lu_panel_reg_kernel<6, PANEL_REG_NT>};
        const int reg_smem = PANEL_REG_ROWS * ((NB + 1) * sizeof(float) + 2 * sizeof(int));
        for (const void* f : reg_kernels)
            VPM_CU(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, reg_smem));
    }
    const size_t solve_smem = (size_t)(n + 32) * sizeof(float);
    VPM_CU(cudaFuncSetAttribute(lu_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)solve_smem));
    // Factor panel k0 on stream ps.
    auto launch_panel = [&](int k0, cudaStream_t ps) {
        const int nb = n - k0 < NB ? n - k0 : NB, rows = n - k0;
        const size_t maps = (size_t)2 * rows * sizeof(int);
        trace_launch();
        if (rows <= PANEL_REG_ROWS) {
            const size_t rsmem = maps + (size_t)rows * (NB + 1) * sizeof(float);
            switch ((rows + PANEL_REG_NT - 1) / PANEL_REG_NT) {
#define VPM_PANEL_R(R)                                                                                              \
    case R:                                                                                                         \
        lu_panel_reg_kernel<R, PANEL_REG_NT><<<1, PANEL_REG_NT, rsmem, ps>>>(LU, n, k0, nb, info, perm, moves); \
        break;
                VPM_PANEL_R(1)
                VPM_PANEL_R(2)
                VPM_PANEL_R(3)
                VPM_PANEL_R(4)
                VPM_PANEL_R(5)
                VPM_PANEL_R(6)
#undef VPM_PANEL_R
            }
            return;
        }
        const int srows = (int)std::min<size_t>(rows, (PANEL_SMEM_MAX - maps) / (PLD * sizeof(float)));
        const size_t psmem = maps + (size_t)srows * PLD * sizeof(float);
        if (srows == rows)
            lu_panel_kernel<true><<<1, PANEL_THREADS, psmem, ps>>>(LU, n, k0, nb, info, perm, moves, pscratch, srows);
        else
            lu_panel_kernel<false><<<1, PANEL_THREADS, psmem, ps>>>(LU, n, k0, nb, info, perm, moves, pscratch, srows);
    };
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int nb = n - k0 < NB ? n - k0 : NB;
        launch_panel(k0, st);
        if (n - nb > 0) {
            trace_launch();
            lu_rows_kernel<<<(n - nb + ROWS_THREADS - 1) / ROWS_THREADS, ROWS_THREADS, 0, st>>>(LU, n, k0, nb, moves);
        }
        const int rest = n - k0 - nb;
        if (rest > 0) {
            trace_launch();
            lu_update_kernel<<<dim3((rest + 63) / 64, (rest + 63) / 64), 256, 0, st>>>(LU, n, k0, nb, k0 + nb, n);
        }
    }
    trace_launch();
    lu_transpose_kernel<<<dim3((n + 31) / 32, (n + 31) / 32), dim3(32, 8), 0, st>>>(LU, T, n);
    VPM_CU(cudaGetLastError());
    int hinfo = 0;
    VPM_CU(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    VPM_CU(cudaStreamSynchronize(st));
    if (hinfo != 0) {
        *msg = "aic_solve: matrix is singular in FP32 (zero pivot)";
        return VPM_ERR_NOT_CONVERGED;
    }
    trace_launch();
    lu_solve_kernel<<<1, LU_THREADS, solve_smem, st>>>(T, perm, n, b, x, 0);
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
        if (iters) *iters = it;
        if (be <= tol) {
            if (berr) *berr = be;
            return VPM_OK;
        }
        const bool last = it >= max_iter || !isfinite(be);
        if (be < best) {  // keep the best iterate (its copy is needed only if another step follows)
            best = be;
            if (!last) VPM_CU(cudaMemcpyAsync(xbest, x, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else if (last && isfinite(best)) {
            VPM_CU(cudaMemcpyAsync(x, xbest, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        if (last) {
            if (berr) *berr = best;
            *msg = "aic_solve: backward error above tol after max_iter refinement steps (best x written)";
            return VPM_ERR_NOT_CONVERGED;
        }
        trace_launch();
        lu_solve_kernel<<<1, LU_THREADS, solve_smem, st>>>(T, perm, n, r, x, 1);
    }
#undef VPM_CU
}

}  // namespace vpm
