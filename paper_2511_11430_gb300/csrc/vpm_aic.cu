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

#include <cooperative_groups.h>

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

// The row-dominant LU's panel and update kernels are launched as programmatic dependents
// of the kernel before them: each lets the next one be scheduled at once and waits,
// before touching the matrix, until the previous grid has completed and its writes
// are visible (griddepcontrol; without the launch attribute both are no-ops).
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// A22 -= L21 U12 over rows [k0+nb, n) and columns [cb, ce): 64x64 output tile per
// block, 4x4 per thread.
__global__ void __launch_bounds__(256) lu_update_kernel(float* __restrict__ A, int n, int k0, int nb, int cb, int ce,
                                                        const float* __restrict__ dsrc)
{
    __shared__ float Ls[64][NB + 1];
    __shared__ float Us[NB][64 + 1];
    pdl_enter();
    if (dsrc && blockIdx.x == 0 && blockIdx.y == 0)  // the panel's factored diagonal block, into place
        for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
            const int i = e / nb, c = e - i * nb;
            A[(size_t)(k0 + i) * n + k0 + c] = dsrc[e];
        }
    const int s0 = k0 + nb;
    const int r0 = s0 + blockIdx.y * 64, c0 = cb + blockIdx.x * 64;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    // this thread's 4 x 4 outputs are read first, so that they arrive with the tiles
    float out[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int r = r0 + ty * 4 + q, c = c0 + tx * 4 + w;
            out[q][w] = (r < n && c < ce) ? A[(size_t)r * n + c] : 0.f;
        }
    for (int e = threadIdx.x; e < 64 * NB; e += blockDim.x) {
        const int i = e / NB, p = e % NB;
        const int r = r0 + i;
        Ls[i][p] = (r < n && p < nb) ? A[(size_t)r * n + k0 + p] : 0.f;
        const int pp = e / 64, cc = e % 64;
        const int c = c0 + cc;
        Us[pp][cc] = (c < ce && pp < nb) ? A[(size_t)(k0 + pp) * n + c] : 0.f;
    }
    __syncthreads();
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
            if (c < ce) A[(size_t)r * n + c] = out[q][w] - acc[q][w];
        }
    }
}

// ---------------------------------------------------------------------------
// LU without row exchanges, for matrices that are strictly diagonally dominant by
// rows (|a_ii| > sum_{j != i} |a_ij| for every i).  Gaussian elimination keeps that
// property in every Schur complement, so no pivot is ever zero and the elements grow
// by at most a factor two: it is stable without pivoting (Wilkinson).  The blade AIC
// systems are of this kind (the self-influence of a ring at its own collocation point
// dominates its row).  Without the pivot search a panel needs no block-wide
// reduction per column: lu_np_panel_kernel factors the 32 x 32 diagonal block in one
// warp and then forms L21 = A21 U11^-1 (one thread per row) and U12 = L11^-1 A12 (one
// thread per column) in parallel over the whole panel; lu_update_kernel follows.
// ---------------------------------------------------------------------------

// LU = A, and flag |= 1 when some row is not strictly diagonally dominant (one warp
// per row, FP64 sums): the copy the factorisation works on and the test in one pass.
__global__ void __launch_bounds__(256) lu_dominance_kernel(const float* __restrict__ A, int n,
                                                           float* __restrict__ LU, int* __restrict__ flag)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    double s = 0.0;
    for (int c = lane; c < n; c += 32) {
        const float a = A[(size_t)i * n + c];
        LU[(size_t)i * n + c] = a;
        s += fabs((double)a);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const double d = fabs((double)A[(size_t)i * n + i]);
        if (!(2.0 * d > s)) atomicOr(flag, 1);
    }
}

constexpr int NP_THREADS = 256;

// Panel [k0, k0 + nb) of the row-dominant LU: grid (chunks, 2); blockIdx.y 0 forms the
// rows of L21 (NP_THREADS rows per block), 1 the columns of U12.  Every block factors
// the diagonal block in shared memory (one warp, no exchanges); block (0, 0) writes it
// to dout (lu_update_kernel copies it into place) or, for the last panel, launched as
// that one block with dout NULL, into A; it also records the first zero or non-finite
// pivot in *info (1-based column) and, for the first panel, sets the permutation to
// the identity and clears *info.
__global__ void __launch_bounds__(NP_THREADS) lu_np_panel_kernel(float* __restrict__ A, int n, int k0, int nb,
                                                                 int* __restrict__ info, int* __restrict__ perm,
                                                                 float* __restrict__ dout)
{
    __shared__ float D[NB][NB + 1];
    __shared__ float Rinv[NB];
    __shared__ float W[NP_THREADS][NB + 1];
    pdl_enter();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool head = blockIdx.x == 0 && blockIdx.y == 0;
    if (head && k0 == 0) {
        for (int i = tid; i < n; i += NP_THREADS) perm[i] = i;
        if (tid == 0) *info = 0;
    }
    const int rest = n - k0 - nb;
    const int base = blockIdx.x * NP_THREADS;
    const int rows = blockIdx.y == 0 ? max(0, min(NP_THREADS, rest - base)) : 0;
    const int col = k0 + nb + base + tid;
    const bool col_ok = blockIdx.y == 1 && base + tid < rest;
    // This block's own part of the panel is requested first, so that it arrives while
    // the diagonal block is factored: the rows of A21 into W (asynchronous copies), the
    // column of A12 into registers.
    for (int e = tid; e < rows * NB; e += NP_THREADS) {
        const int r = e / NB, c = e - r * NB;
        if (c < nb)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(&W[r][c])),
                         "l"(A + (size_t)(k0 + nb + base + r) * n + k0 + c)
                         : "memory");
        else
            W[r][c] = 0.f;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    float y[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) y[i] = (col_ok && i < nb) ? A[(size_t)(k0 + i) * n + col] : 0.f;
    for (int e = tid; e < NB * NB; e += NP_THREADS) {
        const int i = e / NB, c = e - i * NB;
        D[i][c] = (i < nb && c < nb) ? A[(size_t)(k0 + i) * n + k0 + c] : (i == c ? 1.f : 0.f);
    }
    __syncthreads();
    if (warp == 0) {  // D = L11 U11 (unit lower L below the diagonal): lane i holds row i in registers
        float v[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) v[c] = D[lane][c];
#pragma unroll
        for (int j = 0; j < NB - 1; ++j) {
            // one correctly rounded reciprocal of the pivot per step instead of a division
            const float l = v[j] * __frcp_rn(__shfl_sync(0xffffffffu, v[j], j));
#pragma unroll
            for (int c = j + 1; c < NB; ++c) {
                const float u = __shfl_sync(0xffffffffu, v[c], j);  // the pivot row's entry
                if (lane > j) v[c] = fmaf(-l, u, v[c]);
            }
            if (lane > j) v[j] = l;
        }
#pragma unroll
        for (int c = 0; c < NB; ++c) D[lane][c] = v[c];
        Rinv[lane] = __frcp_rn(D[lane][lane]);  // this lane's own diagonal entry
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    if (head) {
        // the factored diagonal block goes to dout (the other blocks of this launch are
        // still reading the original from A), or to A itself when it is the only block
        for (int e = tid; e < nb * nb; e += NP_THREADS) {
            const int i = e / nb, c = e - i * nb;
            if (dout)
                dout[e] = D[i][c];
            else
                A[(size_t)(k0 + i) * n + k0 + c] = D[i][c];
        }
        if (tid < nb) {
            const float d = D[tid][tid];
            if (!(fabsf(d) > 0.f) || !isfinite(d)) atomicCAS(info, 0, k0 + tid + 1);
        }
    }
    if (blockIdx.y == 0) {  // rows of L21: x = a U11^-1 on the rows staged in W
        if (rows <= 0) return;
        if (tid < rows) {
            float x[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) {  // four interleaved partial sums: shorter chains
                float v[4] = {W[tid][j], 0.f, 0.f, 0.f};
#pragma unroll
                for (int p = 0; p < j; ++p) v[p & 3] = fmaf(-x[p], D[p][j], v[p & 3]);
                x[j] = ((v[0] + v[1]) + (v[2] + v[3])) * Rinv[j];
            }
#pragma unroll
            for (int j = 0; j < NB; ++j) W[tid][j] = x[j];
        }
        __syncthreads();
        for (int e = tid; e < rows * NB; e += NP_THREADS) {
            const int r = e / NB, c = e - r * NB;
            if (c < nb) A[(size_t)(k0 + nb + base + r) * n + k0 + c] = W[r][c];
        }
    } else if (col_ok) {  // columns of U12: y = L11^-1 a (unit lower), coalesced across the threads
#pragma unroll
        for (int i = 1; i < NB; ++i) {
            float v[4] = {y[i], 0.f, 0.f, 0.f};
#pragma unroll
            for (int p = 0; p < i; ++p) v[p & 3] = fmaf(-D[i][p], y[p], v[p & 3]);
            y[i] = (v[0] + v[1]) + (v[2] + v[3]);
        }
#pragma unroll
        for (int i = 0; i < NB; ++i)
            if (i < nb) A[(size_t)(k0 + i) * n + col] = y[i];
    }
}

// T = LU^T (32x32 tiles through shared memory), so that the solves read the factors
// column by column with coalesced loads.
__global__ void __launch_bounds__(256) lu_transpose_kernel(const float* __restrict__ LU, float* __restrict__ T,
                                                           int n)
{
    __shared__ float t[32][33];
    pdl_enter();
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

// ---------------------------------------------------------------------------
// Triangular solves on a cluster of SOLVE_CL blocks.  The substitution runs over the
// SB-row diagonal blocks of the factors; the inverse of every diagonal block is formed
// once (lu_diag_inv_kernel), so solving a block is an SB x SB matrix-vector product
// rather than SB dependent steps.  The rows are split into SOLVE_CL contiguous ranges
// of whole SB-row blocks, one per block of the cluster, each of which keeps a full copy
// of the vector in shared memory.  Per diagonal block k: its owner solves it (warps 0
// and 1, one row of the block per thread) and writes the SB values into every block's
// copy (distributed shared memory), one cluster barrier makes them visible, and every
// block subtracts their contribution from its own rows, with the SB factor entries per
// row loaded one step ahead (T = LU^T, so column p of the factors is the contiguous
// row p of T).  One cluster barrier per SB rows bounds the solve's latency; SOLVE_CL
// blocks read the factors from L2 SOLVE_CL times faster than one.
// ---------------------------------------------------------------------------
constexpr int SOLVE_CL = 8;
constexpr int SOLVE_T = 256;
constexpr int SB = 64;

// Inverses of the SB x SB diagonal blocks, transposed: Dinv[(w * nblk + k) * SB * SB + q * SB + i]
// = inverse(block k)[i][q], w = 0 for the unit lower factor L, 1 for the upper U.  One block of
// SB = 64 threads per diagonal block and factor.  Each warp inverts one 32 x 32 diagonal
// sub-block (lane c forms column c by substitution); the off-diagonal sub-block of the
// inverse follows from them by two 32 x 32 products: for L = [[A, 0], [C, B]] it is
// -B^-1 C A^-1, for U = [[A, C], [0, B]] it is -A^-1 C B^-1.  A partial last block is padded
// with the identity.
__global__ void __launch_bounds__(SB) lu_diag_inv_kernel(const float* __restrict__ LU, int n,
                                                         float* __restrict__ Dinv)
{
    static_assert(SB == 64, "two 32 x 32 sub-blocks per diagonal block");
    __shared__ float M[SB][SB + 1];
    __shared__ float Iv[2][32][33];  // inverses of the two diagonal sub-blocks
    __shared__ float Tm[32][33];
    pdl_enter();
    const int k = blockIdx.x, w = blockIdx.y, tid = threadIdx.x, nblk = gridDim.x;
    const int lane = tid & 31, h = tid >> 5;
    const int b0 = SB * k, nb = min(SB, n - b0);
    for (int i = 0; i < SB; ++i)
        M[i][tid] = (i < nb && tid < nb) ? LU[(size_t)(b0 + i) * n + b0 + tid] : (i == tid ? 1.f : 0.f);
    __syncthreads();
    {
        const int o = 32 * h;
        float x[32];
        if (w == 0) {  // L x = e_c, L unit lower: x_i = -sum_{c <= p < i} L[i][p] x_p
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                float v = i == lane ? 1.f : 0.f;
#pragma unroll
                for (int p = 0; p < i; ++p) v = fmaf(-M[o + i][o + p], x[p], v);
                x[i] = i < lane ? 0.f : v;
            }
        } else {  // U x = e_c: x_i = (delta_ic - sum_{i < p <= c} U[i][p] x_p) / U[i][i]
#pragma unroll
            for (int i = 31; i >= 0; --i) {
                float v = i == lane ? 1.f : 0.f;
#pragma unroll
                for (int p = i + 1; p < 32; ++p) v = fmaf(-M[o + i][o + p], x[p], v);
                x[i] = i > lane ? 0.f : v / M[o + i][o + i];
            }
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) Iv[h][i][lane] = x[i];
    }
    __syncthreads();
    // Tm = C A^-1 (L) or C B^-1 (U); thread (h, lane) forms rows 16 h .. 16 h + 15 of column lane
    const int j = lane, ib = 16 * h;
    float s[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) s[q] = 0.f;
#pragma unroll 8
    for (int p = 0; p < 32; ++p) {
        const float ivp = Iv[w][p][j];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            s[q] = fmaf(w == 0 ? M[32 + ib + q][p] : M[ib + q][32 + p], ivp, s[q]);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) Tm[ib + q][j] = s[q];
    __syncthreads();
    // off-diagonal sub-block: -B^-1 Tm (L) or -A^-1 Tm (U)
#pragma unroll
    for (int q = 0; q < 16; ++q) s[q] = 0.f;
#pragma unroll 8
    for (int p = 0; p < 32; ++p) {
        const float tp = Tm[p][j];
#pragma unroll
        for (int q = 0; q < 16; ++q) s[q] = fmaf(-Iv[1 - w][ib + q][p], tp, s[q]);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) Tm[ib + q][j] = s[q];
    __syncthreads();
    float* out = Dinv + ((size_t)w * nblk + k) * SB * SB;
    for (int e = tid; e < SB * SB; e += SB) {  // out[q SB + i] = inverse[i][q]
        const int q = e / SB, i = e % SB;
        float v;
        if ((i < 32) == (q < 32))
            v = Iv[i >= 32][i & 31][q & 31];
        else if (w == 0)
            v = i >= 32 ? Tm[i - 32][q] : 0.f;
        else
            v = i < 32 ? Tm[i][q - 32] : 0.f;
        out[e] = v;
    }
}

// (LU) z = P r in FP32 for a FP64 right-hand side; writes z, or adds it to `out` when
// `accumulate` is set (both FP64).  Launched as one cluster of SOLVE_CL blocks of
// SOLVE_T threads with (n + SB) floats of dynamic shared memory.
__global__ void __cluster_dims__(SOLVE_CL, 1, 1) __launch_bounds__(SOLVE_T)
    lu_solve_cluster_kernel(const float* __restrict__ T, const float* __restrict__ Dinv,
                            const int* __restrict__ perm, int n, const double* __restrict__ rhs,
                            double* __restrict__ out, int accumulate, double* __restrict__ norms)
{
    pdl_enter();
    if (norms && blockIdx.x == 0 && threadIdx.x < 4) norms[threadIdx.x] = 0.0;  // for the residual that follows
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) float y[];  // n entries and SB zeros
    cg::cluster_group cl = cg::this_cluster();
    const int cr = (int)cl.block_rank(), tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nblk = (n + SB - 1) / SB;
    const int per = SB * ((nblk + SOLVE_CL - 1) / SOLVE_CL);  // rows per block of the cluster
    const int r0 = min(n, cr * per), r1 = min(n, r0 + per);
    for (int i = tid; i < n + SB; i += SOLVE_T) y[i] = i < n ? (float)rhs[perm[i]] : 0.f;
    cl.sync();
    const int i0 = r0 + tid;  // this thread's first row (later rows, n > SOLVE_CL SOLVE_T, unprefetched)
    // one direction of the substitution: forward (L, blocks ascending, rows below) or
    // backward (U, blocks descending, rows above)
    auto sweep = [&](bool fwd) {
        const float* Dw = Dinv + (size_t)(fwd ? 0 : nblk) * SB * SB;
        float t[SB];
        auto fetch = [&](int k) {  // row i0's entries of block column k
#pragma unroll
            for (int p = 0; p < SB; ++p) {
                const int c = SB * k + p;
                t[p] = (i0 < r1 && k >= 0 && k < nblk && c < n) ? T[(size_t)c * n + i0] : 0.f;
            }
        };
        float d[SB];  // warps 0 and 1: row 32 warp + lane of the inverse of block k, a step ahead
        auto fetch_d = [&](int k) {
            if (warp < 2 && k >= 0 && k < nblk) {
                const float* Dk = Dw + (size_t)k * SB * SB + 32 * warp + lane;
#pragma unroll
                for (int q = 0; q < SB; ++q) d[q] = Dk[q * SB];
            }
        };
        int k = fwd ? 0 : nblk - 1;
        fetch(k);
        fetch_d(k);
        for (int step = 0; step < nblk; ++step, k += fwd ? 1 : -1) {
            const int b0 = SB * k;
            if (warp < 2 && b0 >= r0 && b0 < r1) {  // this block owns diagonal block k: solve and send
                float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
#pragma unroll
                for (int q = 0; q < SB; q += 4) {
                    v0 = fmaf(d[q], y[b0 + q], v0);
                    v1 = fmaf(d[q + 1], y[b0 + q + 1], v1);
                    v2 = fmaf(d[q + 2], y[b0 + q + 2], v2);
                    v3 = fmaf(d[q + 3], y[b0 + q + 3], v3);
                }
                const float v = (v0 + v1) + (v2 + v3);
                // both warps have read the block before either overwrites it
                asm volatile("bar.sync 1, 64;" ::: "memory");
                const int row = b0 + 32 * warp + lane;
                if (row < n)
                    for (int r = 0; r < SOLVE_CL; ++r) *cl.map_shared_rank(&y[row], r) = v;
            }
            fetch_d(k + (fwd ? 1 : -1));
            cl.sync();
            // subtract block k's contribution from this block's rows beyond it
            const float* yb = y + b0;
            const bool mine = i0 < r1 && (fwd ? i0 >= b0 + SB : i0 < b0);
            float a0 = 0.f, a1 = 0.f;
            if (mine)
#pragma unroll
                for (int p = 0; p < SB; p += 2) {
                    a0 = fmaf(t[p], yb[p], a0);
                    a1 = fmaf(t[p + 1], yb[p + 1], a1);
                }
            fetch(k + (fwd ? 1 : -1));
            if (mine) y[i0] -= a0 + a1;
            for (int i = i0 + SOLVE_T; i < r1; i += SOLVE_T)
                if (fwd ? i >= b0 + SB : i < b0) {
                    float a2 = 0.f;
                    for (int p = 0; p < SB && b0 + p < n; ++p) a2 = fmaf(T[(size_t)(b0 + p) * n + i], yb[p], a2);
                    y[i] -= a2;
                }
            __syncthreads();  // the owner of the next block reads these rows
        }
        cl.sync();
    };
    sweep(true);
    sweep(false);
    for (int i = r0 + tid; i < r1; i += SOLVE_T) out[i] = accumulate ? out[i] + (double)y[i] : (double)y[i];
}

// r = b - A x in FP64 (A's FP32 entries promoted exactly), one warp per row, with the
// row |A| sums stored on the first pass (`first`) and read back on later ones.  The
// maxima of |r_i| (+inf where r_i or x_i is not finite), |x_i|, |b_i| and the row sums
// are folded into out[0..3], zeroed before the launch, by atomic max on their bit
// patterns (non-negative doubles order as their unsigned 64-bit patterns); out[4] and
// out[5] receive the zero-pivot status and the dominance flag.  (The solve before it
// zeroes out[0..3].)
__global__ void __launch_bounds__(256) residual_kernel(const float* __restrict__ A, const double* __restrict__ b,
                                                       const double* __restrict__ x, int n, double* __restrict__ r,
                                                       double* __restrict__ rowabs, int first,
                                                       const int* __restrict__ info, double* __restrict__ out)
{
    __shared__ double red[4][8];
    pdl_enter();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < n) {
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
        const double ri = b[i] - s, xi = x[i];
        if (lane == 0) {
            r[i] = ri;
            if (first) rowabs[i] = a;
        }
        m[0] = isfinite(ri) && isfinite(xi) ? fabs(ri) : INFINITY;
        m[1] = fabs(xi);
        m[2] = fabs(b[i]);
        m[3] = first ? a : rowabs[i];
    }
    if (lane == 0)
        for (int q = 0; q < 4; ++q) red[q][wib] = m[q];
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v = fmax(v, red[threadIdx.x][w]);
        atomicMax(reinterpret_cast<unsigned long long*>(out) + threadIdx.x, (unsigned long long)__double_as_longlong(v));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[4] = (double)info[0], out[5] = (double)info[1];
}

namespace {
struct AicWs {
    size_t lu, t, perm, moves, info, dblk, dinv, pscratch, r, xbest, rowabs, norms, bytes;
};
AicWs aic_layout(int n)
{
    Carve cv;
    AicWs w;
    w.lu = cv.take((size_t)n * n * sizeof(float));
    w.t = cv.take((size_t)n * n * sizeof(float));
    w.perm = cv.take((size_t)n * sizeof(int));
    w.moves = cv.take((1 + 4 * NB) * sizeof(int));
    w.info = cv.take(2 * sizeof(int));  // the factorisation's status, then the dominance test
    w.dblk = cv.take((size_t)NB * NB * sizeof(float));
    w.dinv = cv.take((size_t)2 * ((n + SB - 1) / SB) * SB * SB * sizeof(float));
    w.pscratch = cv.take((size_t)n * PLD * sizeof(float));
    w.r = cv.take((size_t)n * sizeof(double));
    w.xbest = cv.take((size_t)n * sizeof(double));
    w.rowabs = cv.take((size_t)n * sizeof(double));
    w.norms = cv.take(6 * sizeof(double));
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
    float* dblk = reinterpret_cast<float*>(ws + L.dblk);
    float* dinv = reinterpret_cast<float*>(ws + L.dinv);
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
    const size_t solve_smem = (size_t)(n + SB) * sizeof(float);
    VPM_CU(cudaFuncSetAttribute(lu_solve_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)solve_smem));
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
    // Strictly row-dominant matrices (the blade AIC systems) need no row exchanges
    // (Gaussian elimination keeps them dominant, with growth at most 2), so the LU
    // without them runs first and the dominance test is read with the first
    // residual: any other matrix is then factored again with partial pivoting.  The
    // zero-pivot status is read at the same synchronisation.
    int* dflag = info + 1;
    // Kernels after the first are launched as programmatic dependents (pdl_enter).
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    auto cfg = [&](dim3 g, dim3 b, size_t smem = 0) {
        cudaLaunchConfig_t c = {};
        c.gridDim = g;
        c.blockDim = b;
        c.dynamicSmemBytes = smem;
        c.stream = st;
        c.attrs = pdl;
        c.numAttrs = 1;
        return c;
    };
    auto factor = [&](bool pivot) -> cudaError_t {
        for (int k0 = 0; !pivot && k0 < n; k0 += NB) {
            const int nb = n - k0 < NB ? n - k0 : NB;
            const int rest = n - k0 - nb;
            trace_launch();
            cudaError_t e;
            if (rest > 0) {
                const cudaLaunchConfig_t c = cfg(dim3((rest + NP_THREADS - 1) / NP_THREADS, 2), dim3(NP_THREADS));
                e = cudaLaunchKernelEx(&c, lu_np_panel_kernel, LU, n, k0, nb, info, perm, dblk);
            } else {
                const cudaLaunchConfig_t c = cfg(dim3(1, 1), dim3(NP_THREADS));
                e = cudaLaunchKernelEx(&c, lu_np_panel_kernel, LU, n, k0, nb, info, perm, (float*)nullptr);
            }
            if (e != cudaSuccess) return e;
            if (rest > 0) {
                trace_launch();
                const cudaLaunchConfig_t c = cfg(dim3((rest + 63) / 64, (rest + 63) / 64), dim3(256));
                e = cudaLaunchKernelEx(&c, lu_update_kernel, LU, n, k0, nb, k0 + nb, n, (const float*)dblk);
                if (e != cudaSuccess) return e;
            }
        }
        for (int k0 = 0; pivot && k0 < n; k0 += NB) {
            const int nb = n - k0 < NB ? n - k0 : NB;
            launch_panel(k0, st);
            if (n - nb > 0) {
                trace_launch();
                lu_rows_kernel<<<(n - nb + ROWS_THREADS - 1) / ROWS_THREADS, ROWS_THREADS, 0, st>>>(LU, n, k0, nb,
                                                                                                    moves);
            }
            const int rest = n - k0 - nb;
            if (rest > 0) {
                trace_launch();
                lu_update_kernel<<<dim3((rest + 63) / 64, (rest + 63) / 64), 256, 0, st>>>(LU, n, k0, nb, k0 + nb,
                                                                                           n, nullptr);
            }
        }
        trace_launch(3);
        cudaError_t e;
        {
            const cudaLaunchConfig_t c = cfg(dim3((n + 31) / 32, (n + 31) / 32), dim3(32, 8));
            if ((e = cudaLaunchKernelEx(&c, lu_transpose_kernel, (const float*)LU, T, n)) != cudaSuccess) return e;
        }
        {
            const cudaLaunchConfig_t c = cfg(dim3((n + SB - 1) / SB, 2), dim3(SB));
            if ((e = cudaLaunchKernelEx(&c, lu_diag_inv_kernel, (const float*)LU, n, dinv)) != cudaSuccess) return e;
        }
        {
            const cudaLaunchConfig_t c = cfg(dim3(SOLVE_CL), dim3(SOLVE_T), solve_smem);
            e = cudaLaunchKernelEx(&c, lu_solve_cluster_kernel, (const float*)T, (const float*)dinv, (const int*)perm,
                                   n, b, x, 0, norms);
        }
        return e != cudaSuccess ? e : cudaGetLastError();
    };
    VPM_CU(cudaMemsetAsync(dflag, 0, sizeof(int), st));
    trace_launch();
    lu_dominance_kernel<<<(n * 32 + 255) / 256, 256, 0, st>>>(A, n, LU, dflag);
    VPM_CU(factor(false));
    bool pivoted = false;
    double h[6];
    double best = INFINITY;
    for (int it = 0;; ++it) {
        trace_launch();
        {
            const cudaLaunchConfig_t c = cfg(dim3((n * 32 + 255) / 256), dim3(256));
            VPM_CU(cudaLaunchKernelEx(&c, residual_kernel, A, (const double*)b, (const double*)x, n, r, rowabs,
                                      it == 0 ? 1 : 0, (const int*)info, norms));
        }
        VPM_CU(cudaGetLastError());
        VPM_CU(cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, st));
        VPM_CU(cudaStreamSynchronize(st));
        if (!pivoted && h[5] != 0.0) {  // not row-dominant: factor again with row exchanges
            pivoted = true;
            VPM_CU(cudaMemcpyAsync(LU, A, (size_t)n * n * sizeof(float), cudaMemcpyDeviceToDevice, st));
            VPM_CU(factor(true));
            it = -1;
            continue;
        }
        if (h[4] != 0.0) {
            *msg = "aic_solve: matrix is singular in FP32 (zero pivot)";
            return VPM_ERR_NOT_CONVERGED;
        }
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
        {
            const cudaLaunchConfig_t c = cfg(dim3(SOLVE_CL), dim3(SOLVE_T), solve_smem);
            VPM_CU(cudaLaunchKernelEx(&c, lu_solve_cluster_kernel, (const float*)T, (const float*)dinv,
                                      (const int*)perm, n, (const double*)r, x, 1, norms));
        }
    }
#undef VPM_CU
}

}  // namespace vpm
