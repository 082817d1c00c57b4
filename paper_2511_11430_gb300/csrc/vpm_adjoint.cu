// Adjoint of the Gaussian-particle velocity at a set of evaluation points.
//
// Forward: u_k = sum_j K(r) Gamma_j x r, r = y_k - x_j (Eq. 2-4).  Given the loss
// gradient g_k = dL/du_k, the chain rule gives for every particle j
//   dL/dGamma_j = sum_k K (r x g_k)
//   dL/dx_j     = sum_k [K (Gamma_j x g_k) - H ((Gamma_j x r) . g_k) r]
//              = Gamma_j x W_j + 3/(4 pi) sum_k h ((Gamma_j x r) . g_k) r,
// with W_j = sum_k K g_k, H = K'(r)/r = -3 h/(4 pi) and the 1/(4 pi) of K taken out
// of the sums.  Every pair term is recomputed; nothing of the forward is stored.
//
// The kernel mirrors the forward sweep with the roles swapped: a thread owns two
// particles (packed lanes), the evaluation points and their g_k stream through
// shared memory in 128-point tiles (bulk copies, double-buffered), work is split
// stream-K over (particle tile, point tile) pairs and the partial sums are reduced
// in a fixed order by a second kernel that also forms the outputs.
#include <math.h>

#include "vpm_common.cuh"
#include "vpm_internal.h"
#include "vpm_kernel.cuh"

namespace vpm {

constexpr int A_F4 = 5;  // float4 per packed evaluation point
constexpr int A_NC = 9;  // accumulators: dG (3), W (3), X3 (3)
constexpr uint64_t A_WAIT_LIMIT = 2000000000ull;  // 2 s of wall time

// Packed point (both lanes equal): (yx,yx,yy,yy) (yz,yz,gx,gx) (gy,gy,gz,gz) (-gx,-gx,-gy,-gy) (-gz,-gz,0,0)
__global__ void __launch_bounds__(SRC_TILE) pack_points_kernel(const float4* __restrict__ tgt,
                                                               const float* __restrict__ g, int n,
                                                               float4* __restrict__ out, float4* __restrict__ box)
{
    const int k = blockIdx.x * SRC_TILE + threadIdx.x;
    const bool valid = k < n;
    float x = 0.f, y = 0.f, z = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    if (valid) {
        const float4 p = tgt[k];
        x = p.x, y = p.y, z = p.z;
        gx = g[k], gy = g[n + k], gz = g[2 * n + k];
    }
    float4* o = out + (size_t)k * A_F4;
    o[0] = make_float4(x, x, y, y);
    o[1] = make_float4(z, z, gx, gx);
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

struct AdjAcc {
    f2 v[A_NC];  // dG x,y,z | W x,y,z | X3 x,y,z
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < A_NC; ++i) v[i] = zero2();
    }
};

template <bool NEAR>
__device__ __forceinline__ void adjoint_tile(AdjAcc& a, const float4* __restrict__ s, int cnt, f2 NX, f2 NY, f2 NZ,
                                             f2 GX, f2 GY, f2 GZ, f2 NGX, f2 NGY, f2 NGZ, const NearConst& nc)
{
#pragma unroll 2
    for (int j = 0; j < cnt; ++j) {
        const float4* e = s + j * A_F4;
        const float4 q0 = e[0], q1 = e[1], q2 = e[2], q3 = e[3], q4 = e[4];
        const f2 gx = make_float2(q1.z, q1.w), gy = make_float2(q2.x, q2.y), gz = make_float2(q2.z, q2.w);
        const f2 ngx = make_float2(q3.x, q3.y), ngy = make_float2(q3.z, q3.w), ngz = make_float2(q4.x, q4.y);
        const f2 rx = add2(make_float2(q0.x, q0.y), NX);  // y_k - x_j
        const f2 ry = add2(make_float2(q0.z, q0.w), NY);
        const f2 rz = add2(make_float2(q1.x, q1.y), NZ);
        const f2 r2 = fma2(rz, rz, fma2(ry, ry, mul2(rx, rx)));
        f2 K, h;
        if (NEAR) {
            near_kh(r2.x, nc, K.x, h.x);
            near_kh(r2.y, nc, K.y, h.y);
        } else {
            const f2 rs = rsqrt2_approx(r2);
            const f2 i2 = mul2(rs, rs);
            K = mul2(i2, rs);
            h = mul2(K, i2);
        }
        // dG += K (r x g)
        a.v[0] = fma2(K, fma2(ry, gz, mul2(rz, ngy)), a.v[0]);
        a.v[1] = fma2(K, fma2(rz, gx, mul2(rx, ngz)), a.v[1]);
        a.v[2] = fma2(K, fma2(rx, gy, mul2(ry, ngx)), a.v[2]);
        // W += K g
        a.v[3] = fma2(K, gx, a.v[3]);
        a.v[4] = fma2(K, gy, a.v[4]);
        a.v[5] = fma2(K, gz, a.v[5]);
        // c = Gamma_j x r, t = c . g, X3 += h t r
        const f2 cx = fma2(GY, rz, mul2(NGZ, ry));
        const f2 cy = fma2(GZ, rx, mul2(NGX, rz));
        const f2 cz = fma2(GX, ry, mul2(NGY, rx));
        const f2 ht = mul2(h, fma2(cz, gz, fma2(cy, gy, mul2(cx, gx))));
        a.v[6] = fma2(ht, rx, a.v[6]);
        a.v[7] = fma2(ht, ry, a.v[7]);
        a.v[8] = fma2(ht, rz, a.v[8]);
    }
}

struct AdjArgs {
    const float4* pos;
    const float4* str;
    int n_src;
    const float4* pts;  // packed points
    const float4* pbox;
    int n_pts;
    StreamK sk;
    NearConst nc;
    float* part;
    int* dev_err;
};

template <bool COMP>
__global__ void __launch_bounds__(TPB, 1) adjoint_kernel(const AdjArgs A)
{
    constexpr int BUF = SRC_TILE * A_F4;
    __shared__ __align__(128) float4 sbuf[2][BUF];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ float wbox[TPB / 32][12];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const StreamK& sk = A.sk;
    const int b = blockIdx.x;
    const long long lo_b = sk.lo(b), hi_b = sk.lo(b + 1);
    int t, k;
    sk.first_at_or_after(lo_b, t, k);
    if (t >= sk.TT || sk.unit_start(t, k) >= hi_b) return;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int kk, int slot) {
        fence_proxy_async_smem();
        mbar_expect_tx(&bars[slot], BUF * 16);
        bulk_g2s(&sbuf[slot][0], A.pts + (size_t)kk * BUF, BUF * 16, &bars[slot]);
    };
    if (tid == 0) issue(k, 0);

    AdjAcc acc, hi, lo;
    acc.zero();
    if (COMP) {
        hi.zero();
        lo.zero();
    }
    f2 NX = zero2(), NY = zero2(), NZ = zero2(), GX = zero2(), GY = zero2(), GZ = zero2();
    int cur_t = -1;
    uint32_t ph0 = 0, ph1 = 0;
    bool outstanding = false;
    for (int it = 0;; ++it) {
        const int slot = it & 1;
        int nt = t, nk = k + 1;
        if (nk == sk.np) {
            nk = 0;
            ++nt;
        }
        const bool has_next = nt < sk.TT && sk.unit_start(nt, nk) < hi_b;
        if (has_next && tid == 0) issue(nk, slot ^ 1);
        outstanding = has_next;
        if (t != cur_t) {
            cur_t = t;
            const int i0 = t * ADJ_TILE + warp * 64 + lane, i1 = i0 + 32;
            const bool v0 = i0 < A.n_src, v1 = i1 < A.n_src;
            float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0, g0 = p0, g1 = p0;
            if (v0) p0 = A.pos[i0], g0 = A.str[i0];
            if (v1) p1 = A.pos[i1], g1 = A.str[i1];
            NX = make_float2(-p0.x, -p1.x);
            NY = make_float2(-p0.y, -p1.y);
            NZ = make_float2(-p0.z, -p1.z);
            GX = make_float2(g0.x, g1.x);
            GY = make_float2(g0.y, g1.y);
            GZ = make_float2(g0.z, g1.z);
            warp_two_boxes(make_float3(p0.x, p0.y, p0.z), v0, make_float3(p1.x, p1.y, p1.z), v1, wbox[warp]);
        }
        const bool ok = mbar_wait_bounded(&bars[slot], slot ? ph1 : ph0, A.dev_err, A_WAIT_LIMIT);
        if (slot)
            ph1 ^= 1;
        else
            ph0 ^= 1;
        if (!__syncthreads_and(ok)) break;

        const float4* s = &sbuf[slot][0];
        const int cnt = min(SRC_TILE, A.n_pts - k * SRC_TILE);
        const float4 tlo = A.pbox[2 * k], thi = A.pbox[2 * k + 1];
        const f2 NGX = mul2(GX, splat(-1.f)), NGY = mul2(GY, splat(-1.f)), NGZ = mul2(GZ, splat(-1.f));
        if (boxes_near(wbox[warp], tlo, thi, A.nc.far2))
            adjoint_tile<true>(acc, s, cnt, NX, NY, NZ, GX, GY, GZ, NGX, NGY, NGZ, A.nc);
        else
            adjoint_tile<false>(acc, s, cnt, NX, NY, NZ, GX, GY, GZ, NGX, NGY, NGZ, A.nc);
        if (COMP) {
#pragma unroll
            for (int i = 0; i < A_NC; ++i) fold2(hi.v[i], lo.v[i], acc.v[i]);
            acc.zero();
        }
        __syncthreads();
        if (!has_next || nt != t) {
            float* P = A.part + ((size_t)(b + t) * (COMP ? 2 * A_NC : A_NC)) * ADJ_TILE + warp * 64 + lane;
#pragma unroll
            for (int i = 0; i < A_NC; ++i) {
                const f2 v = COMP ? hi.v[i] : acc.v[i];
                P[(size_t)i * ADJ_TILE] = v.x;
                P[(size_t)i * ADJ_TILE + 32] = v.y;
                if (COMP) {
                    P[(size_t)(A_NC + i) * ADJ_TILE] = lo.v[i].x;
                    P[(size_t)(A_NC + i) * ADJ_TILE + 32] = lo.v[i].y;
                }
            }
            acc.zero();
            if (COMP) {
                hi.zero();
                lo.zero();
            }
        }
        if (!has_next) {
            outstanding = false;
            break;
        }
        t = nt;
        k = nk;
    }
    if (outstanding && tid == 0) {
        mbar_wait_bounded(&bars[0], ph0, A.dev_err, A_WAIT_LIMIT);
        mbar_wait_bounded(&bars[1], ph1, A.dev_err, A_WAIT_LIMIT);
    }
}

struct AdjEpiArgs {
    StreamK sk;
    const float* part;
    const float4* str;
    int n, comp;
    float* dx;
    float* dG;
};

__global__ void __launch_bounds__(256) adjoint_epilogue_kernel(const AdjEpiArgs E)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= E.n) return;
    const StreamK& sk = E.sk;
    const int t = i / ADJ_TILE, l = i % ADJ_TILE;
    // partial sums folded in FP32 double-float (two-sum), converted to FP64 once per row
    float H[A_NC], Lw[A_NC];
#pragma unroll
    for (int c = 0; c < A_NC; ++c) H[c] = 0.f, Lw[c] = 0.f;
    if (sk.np > 0) {
        const int b0 = sk.block_of(sk.unit_start(t, 0));
        const int b1 = sk.block_of(sk.unit_start(t, sk.np - 1));
        const int rows = E.comp ? 2 * A_NC : A_NC;
        for (int b = b0; b <= b1; ++b) {
            const long long lo_b = sk.lo(b), hi_b = sk.lo(b + 1);
            const long long c0 = lo_b > (long long)t * sk.C ? lo_b : (long long)t * sk.C;
            int tt, kk;
            sk.first_at_or_after(c0, tt, kk);
            if (tt != t || sk.unit_start(tt, kk) >= hi_b) continue;
            const float* P = E.part + (size_t)(b + t) * rows * ADJ_TILE + l;
#pragma unroll
            for (int c = 0; c < A_NC; ++c) {
                float sum, err;
                two_sum(H[c], P[(size_t)c * ADJ_TILE], sum, err);
                H[c] = sum;
                Lw[c] = __fadd_rn(Lw[c], err);
                if (E.comp) Lw[c] = __fadd_rn(Lw[c], P[(size_t)(A_NC + c) * ADJ_TILE]);
            }
        }
    }
    double acc[A_NC];
#pragma unroll
    for (int c = 0; c < A_NC; ++c) acc[c] = (double)H[c] + (double)Lw[c];
    const double f4pi = 0.079577471545947667884;
    const float4 g = E.str[i];
    const double Gx = g.x, Gy = g.y, Gz = g.z;
    const double Wx = acc[3], Wy = acc[4], Wz = acc[5];
    E.dG[i] = (float)(acc[0] * f4pi);
    E.dG[E.n + i] = (float)(acc[1] * f4pi);
    E.dG[2 * E.n + i] = (float)(acc[2] * f4pi);
    E.dx[i] = (float)((Gy * Wz - Gz * Wy + 3.0 * acc[6]) * f4pi);
    E.dx[E.n + i] = (float)((Gz * Wx - Gx * Wz + 3.0 * acc[7]) * f4pi);
    E.dx[2 * E.n + i] = (float)((Gx * Wy - Gy * Wx + 3.0 * acc[8]) * f4pi);
}

namespace {
struct AdjPlan {
    StreamK sk;
    size_t off_pts, off_box, off_part, bytes;
};

template <bool C>
int adj_occ()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, adjoint_kernel<C>, TPB, 0) != cudaSuccess) nb = 1;
    return nb < 1 ? 1 : nb;
}

AdjPlan plan_adjoint(int64_t n_src, int64_t n_tgt, bool comp)
{
    AdjPlan p;
    StreamK& sk = p.sk;
    sk.TT = (int)((n_src + ADJ_TILE - 1) / ADJ_TILE);
    sk.np = (int)((n_tgt + SRC_TILE - 1) / SRC_TILE);
    sk.ns = 0;
    sk.wp = 1;
    sk.ws = 1;
    sk.C = sk.np;
    sk.tot = (long long)sk.TT * sk.C;
    long long B = (long long)adjoint_blocks(comp);
    if (B > sk.tot) B = sk.tot;
    if (B < 1) B = 1;
    sk.B = (int)B;
    Carve cv;
    p.off_pts = cv.take((size_t)sk.np * SRC_TILE * A_F4 * 16);
    p.off_box = cv.take((size_t)sk.np * 2 * 16);
    p.off_part = cv.take((size_t)(sk.TT + sk.B) * (comp ? 2 : 1) * A_NC * ADJ_TILE * sizeof(float));
    p.bytes = cv.off;
    return p;
}
}  // namespace

int adjoint_blocks(bool comp)
{
    const int sms = sm_count();
    return (comp ? adj_occ<true>() : adj_occ<false>()) * (sms > 0 ? sms : 1);
}

size_t backward_workspace(int64_t n_src, int64_t n_tgt, bool comp)
{
    return plan_adjoint(n_src, n_tgt, comp).bytes;
}

cudaError_t run_backward(char* ws, size_t ws_bytes, const float* src_pos, const float* src_str, int n_src,
                         const float* tgt, int n_tgt, float sigma, bool comp, const float* g, float* dx, float* dG,
                         cudaStream_t st)
{
    if (n_src == 0) return cudaSuccess;
    if (n_tgt == 0) {
        cudaMemsetAsync(dx, 0, sizeof(float) * 3 * (size_t)n_src, st);
        cudaMemsetAsync(dG, 0, sizeof(float) * 3 * (size_t)n_src, st);
        return cudaGetLastError();
    }
    const AdjPlan p = plan_adjoint(n_src, n_tgt, comp);
    if (p.bytes > ws_bytes) return cudaErrorInvalidValue;
    float4* pts = reinterpret_cast<float4*>(ws + p.off_pts);
    float4* box = reinterpret_cast<float4*>(ws + p.off_box);
    float* part = reinterpret_cast<float*>(ws + p.off_part);
    trace_launch();
    pack_points_kernel<<<p.sk.np, SRC_TILE, 0, st>>>(reinterpret_cast<const float4*>(tgt), g, n_tgt, pts, box);
    AdjArgs A;
    A.pos = reinterpret_cast<const float4*>(src_pos);
    A.str = reinterpret_cast<const float4*>(src_str);
    A.n_src = n_src;
    A.pts = pts;
    A.pbox = box;
    A.n_pts = n_tgt;
    A.sk = p.sk;
    const double s = sigma;
    A.nc.inv_s2 = (float)(1.0 / (s * s));
    A.nc.inv_s3 = (float)(1.0 / (s * s * s));
    A.nc.inv_s5 = (float)(1.0 / (s * s * s * s * s));
    A.nc.far2 = (float)((double)RHO_FAR * RHO_FAR * s * s);
    A.part = part;
    A.dev_err = dev_err_ptr();
    {
        TraceScope ts(VPM_TRACE_ADJOINT, st);
        if (comp)
            adjoint_kernel<true><<<p.sk.B, TPB, 0, st>>>(A);
        else
            adjoint_kernel<false><<<p.sk.B, TPB, 0, st>>>(A);
    }
    AdjEpiArgs E;
    E.sk = p.sk;
    E.part = part;
    E.str = reinterpret_cast<const float4*>(src_str);
    E.n = n_src;
    E.comp = comp ? 1 : 0;
    E.dx = dx;
    E.dG = dG;
    trace_launch();
    adjoint_epilogue_kernel<<<(n_src + 255) / 256, 256, 0, st>>>(E);
    return cudaGetLastError();
}

}  // namespace vpm
