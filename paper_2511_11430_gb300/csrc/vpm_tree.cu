// Treecode evaluation of the particle velocity and velocity gradient (Eq. 2-4) of n
// particles on themselves, in O(n log n) work: the fast summation that Sec. II.B
// calls for in place of the direct sum (the paper uses a Cartesian FMM; this is a
// Cartesian Taylor treecode with cluster-to-leaf local expansions: the FMM's
// expansions without their translations between tree levels).
//
// Tree.  The particles are sorted along a Morton (Z-order) curve of their positions
// (21 bits per axis) and the sorted array is halved recursively: node (l, k) of
// level l holds the particles [floor(k n / 2^l), floor((k + 1) n / 2^l)), so every
// node is one contiguous run of the sorted array, node i has children 2i + 1 and
// 2i + 2, and the leaves (level D) hold 33 to 64 particles.  A node carries the
// centre c of its bounding box, the radius r of a sphere about c that holds its
// particles, and its scaled moments M_k = sum_j Gamma_j (x_j - c)^k / k! for the
// multi-indices |k| <= p (k! = k1! k2! k3!, d^k = d1^k1 d2^k2 d3^k3).
//
// Expansion.  Beyond 7 sigma the blob kernel is the point-vortex kernel to FP32
// precision, and u = curl Psi / (4 pi) with Psi(x) = sum_j Gamma_j / |x - x_j|.
// With R = x - c and d_j = x_j - c, Taylor expansion in d_j gives
//   Psi^l(x) = sum_k M_k^l b_k(R),  b_k = (-1)^|k| d^k(1/|R|)/dR^k,  |k| <= p,
// and d b_k / dR_j = -b_{k + e_j}.  The b_k follow from b_0 = 1/|R| by the
// recurrence of the derivatives of 1/|R|,
//   |k| |R|^2 b_k = (2|k| - 1) sum_i k_i R_i b_{k - e_i} - (|k| - 1) sum_i k_i (k_i - 1) b_{k - 2 e_i}
// (the Taylor-coefficient recurrence of 1/|x - y| with the factorials moved into b_k).
// Moving a node's moments from a child centre c' to the parent centre c is the
// product of two truncated series: M_k = sum_{i <= k} M'_i s^(k - i) / (k - i)!,
// s = c' - c.  A far cluster s acts on a target leaf t (centre c_t, x = c_t + y,
// R0 = c_t - c_s) through the leaf's local expansion of order q = p + 1,
//   Psi^l(c_t + y) = sum_{|m| <= q} L_m^l y^m / m!,  L_m^l = (-1)^|m| sum_k M_k^l b_{k + m}(R0),
// summed over every far cluster of the leaf, and at each target
//   4 pi u_a = eps_ajl sum_m L^l_{m + e_j} y^m / m!,   4 pi (grad u)_ab = eps_ajl sum_m L^l_{m + e_j + e_b} y^m / m!.
//
// Traversal.  One warp per target leaf (its targets two per thread, in the lanes of
// packed float2 registers, as in the direct sweep) walks the tree depth first from
// the root with its stack spread over the warp's lanes.  A node is far from the
// leaf when r_node + r_leaf < theta |c_node - c_leaf| and every pair is at least
// 7 sigma apart; a far node enters the leaf's local expansion (the warp computes
// the b_k(R0) together, order by order, into a dense table in shared memory, and
// each lane accumulates its share of the L_m), a leaf that is not far enters by the
// direct sum with the regularised kernel, and any other node is opened.  After the
// walk every target evaluates the local expansion once.  theta = 0 opens every
// node, which gives the direct sum.
//
// Right-hand side (vpm_rhs_tree).  The segments form a second source tree that every
// target leaf walks after the particle tree (far nodes into the same local expansion,
// the others by the exact segment kernel); the summed u and grad u give Vreman's eddy
// viscosity, the stretching and dx/dt per particle; the PSE term of Eq. 5 is then
// summed by a second walk of the particle tree that visits only the nodes within
// 7 sigma of each target leaf.
#include <math.h>

#include <algorithm>
#include <mutex>

#include <cub/device/device_radix_sort.cuh>

#include "vpm_common.cuh"
#include "vpm_internal.h"
#include "vpm_kernel.cuh"

namespace vpm {
namespace {

constexpr int TREE_LEAF = 64;        // particles per leaf at most: one warp's targets
constexpr int TREE_WARPS = 8;        // warps per traversal block
constexpr int TREE_STAGE = 64;       // sources staged in shared memory at a time: a whole leaf
static_assert(TREE_STAGE == 32 || TREE_STAGE == 64, "one or two warp-wide masks per staged run");
constexpr int TREE_MAX_P = 4;        // highest expansion order
constexpr int BOUNDS_BLOCKS = 1024;  // partial boxes of the bounding-box pass
constexpr int MORTON_BITS = 21;      // per axis

__host__ __device__ constexpr int nterms(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// Position of the multi-index (a, b, c) in the graded order: by |k|, then a
// descending, then b descending.
__host__ __device__ constexpr int midx(int a, int b, int c)
{
    return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}

int tree_depth(long long n)
{
    int D = 0;
    while (((n + (1LL << D) - 1) >> D) > TREE_LEAF) ++D;
    return D;
}

// Smallest particle count of a far node that enters the leaf's local expansion:
// below it the point-vortex sum over its particles is cheaper (about 16 lane
// operations per pair and target against about 1,000 per lane for the expansion).
constexpr int M2L_MIN = 32;

// ---------------------------------------------------------------------------
// Near-field blob functions by table.  With x = rho^2 / 2, the direct sweep's kernel
// functions are q(x) = g / rho^3 = 2^(-3/2) e^(-x) sum_k x^k / Gamma(k + 5/2) and
// f = dq/dx = -(3/2) 2^(-3/2) e^(-x) sum_k x^k / Gamma(k + 7/2), whose derivative is
// f' = (15/4) 2^(-3/2) e^(-x) sum_k x^k / Gamma(k + 9/2): the derivative of
// e^(-x) sum_k x^k / Gamma(k + a) is e^(-x) sum_k x^k ((k + 1) c_{k+1} - c_k) with
// c_k = 1 / Gamma(k + a), that is -(a - 1) e^(-x) sum_k x^k / Gamma(k + a + 1).  All
// three series have positive terms, so on the host in FP64 they are exact to rounding
// for every x up to 24.5 (rho = 7).  The treecode's near pairs interpolate q (with
// q' = f) and f (with f') by cubic Hermite polynomials on NEAR_NT equal intervals of
// x: the interpolation error is far below FP32 rounding, and a pair costs two table
// reads and a few FMAs instead of the series or the erf form with their per-lane
// branches.
// ---------------------------------------------------------------------------
constexpr int NEAR_NT = 1024;
constexpr float NEAR_XMAX = 0.5f * RHO_FAR * RHO_FAR;

static __device__ float4 g_near_table[NEAR_NT + 1];  // (q, D f, f, D f') at x_i = i D, D = NEAR_XMAX / NEAR_NT

void near_table_host(float4* t)
{
    const double D = (double)NEAR_XMAX / NEAR_NT, c = 0.35355339059327376;  // 2^(-3/2)
    for (int i = 0; i <= NEAR_NT; ++i) {
        const double x = i * D;
        double term = 4.0 / (3.0 * sqrt(3.14159265358979323846));  // x^k / Gamma(k + 5/2), k = 0
        double T = 0.0, U = 0.0, V = 0.0;
        for (int k = 0; k < 400; ++k) {
            const double u = term / (k + 2.5), v = u / (k + 3.5);  // x^k / Gamma(k + 7/2), x^k / Gamma(k + 9/2)
            T += term, U += u, V += v;
            if (k > 10 && term < 1e-18 * T) break;
            term *= x / (k + 2.5);
        }
        const double e = c * exp(-x);
        const double q = e * T, f = -1.5 * e * U, fp = 3.75 * e * V;
        t[i] = make_float4((float)q, (float)(D * f), (float)f, (float)(D * fp));
    }
}

std::mutex g_near_mu;
bool g_near_ready[64];

// Uploads the table to the current device once (a synchronous copy).
cudaError_t near_table_ready()
{
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_near_mu);
    if (g_near_ready[d]) return cudaSuccess;
    static float4 host[NEAR_NT + 1];
    static bool built = false;
    if (!built) near_table_host(host), built = true;
    e = cudaMemcpyToSymbol(g_near_table, host, sizeof(host));
    if (e == cudaSuccess) g_near_ready[d] = true;
    return e;
}

// K (without 1/(4 pi)) and h = H (-1/3) (without 1/(4 pi)) of one pair, as near_kh,
// with the regularised part from the table T (in shared memory).  Branch-free: every
// lane takes both the table and the point-vortex form and keeps one, so that lanes on
// either side of 7 sigma do not split the warp (measured 2-5% faster than branching).
__device__ __forceinline__ void near_kh_table(float r2, const NearConst& nc, const float4* __restrict__ T, float& K,
                                              float& h)
{
    const bool far = r2 >= nc.far2, zero = r2 == 0.f;
    const float rs = rsqrt_approx(r2);
    const float i2 = rs * rs;
    const float Kf = i2 * rs, hf = Kf * i2;
    // the table's interval (clamped to the last one beyond 7 sigma, where it is not used)
    const float t = fminf((0.5f * r2 * nc.inv_s2) * ((float)NEAR_NT / NEAR_XMAX), (float)NEAR_NT);
    const int i = min((int)t, NEAR_NT - 1);
    const float s = t - (float)i;
    const float4 a = T[i], b = T[i + 1];
    const float s2 = s * s, s3 = s2 * s;
    const float h01 = fmaf(-2.f, s3, 3.f * s2);  // cubic Hermite basis
    const float h00 = 1.f - h01;
    const float h10 = fmaf(-2.f, s2, s3 + s);
    const float h11 = s3 - s2;
    const float q = fmaf(h00, a.x, fmaf(h10, a.y, fmaf(h01, b.x, h11 * b.y)));
    const float f = fmaf(h00, a.z, fmaf(h10, a.w, fmaf(h01, b.z, h11 * b.w)));
    K = zero ? 0.f : (far ? Kf : q * nc.inv_s3);
    h = zero ? 0.f : (far ? hf : f * (-1.0f / 3.0f) * nc.inv_s5);
}

// One source against the thread's two targets with the tabulated near kernel.
template <bool GRAD>
__device__ __forceinline__ void near_source_table(Acc<GRAD, false>& a, const float4* __restrict__ e, f2 X, f2 Y,
                                                  f2 Z, const NearConst& nc, const float4* __restrict__ T)
{
    const float4 q0 = e[0], q1 = e[1], q2 = e[2], q3 = e[3], q4 = e[4];
    const f2 rx = add2(X, make_float2(q0.x, q0.y));
    const f2 ry = add2(Y, make_float2(q0.z, q0.w));
    const f2 rz = add2(Z, make_float2(q1.x, q1.y));
    const f2 r2 = fma2(rz, rz, fma2(ry, ry, mul2(rx, rx)));
    f2 K, h;
    near_kh_table(r2.x, nc, T, K.x, h.x);
    near_kh_table(r2.y, nc, T, K.y, h.y);
    accum_particle<GRAD, false, true>(a, K, h, rx, ry, rz, make_float2(q1.z, q1.w), make_float2(q2.x, q2.y),
                                      make_float2(q2.z, q2.w), make_float2(q3.x, q3.y), make_float2(q3.z, q3.w),
                                      make_float2(q4.x, q4.y), Own{});
}

struct TreeWs {
    size_t part, keys0, keys1, idx0, idx1, cub, cub_bytes, psrc, geo, box, mom, counter, lkey0, lkey1, lord0,
        lord1, bytes;
    int D;
    long long nodes;
};

// The layout of the workspace; fails only if the sort's scratch query does.
cudaError_t tree_layout(long long n, TreeWs& w)
{
    Carve cv;
    w = TreeWs{};
    w.D = tree_depth(n);
    w.nodes = (2LL << w.D) - 1;
    w.part = cv.take((size_t)(BOUNDS_BLOCKS + 1) * 6 * sizeof(float));
    w.keys0 = cv.take((size_t)n * 8);
    w.keys1 = cv.take((size_t)n * 8);
    w.idx0 = cv.take((size_t)n * 4);
    w.idx1 = cv.take((size_t)n * 4);
    size_t cb = 0;
    const cudaError_t e = cub::DeviceRadixSort::SortPairs(
        nullptr, cb, (const unsigned long long*)nullptr, (unsigned long long*)nullptr, (const int*)nullptr,
        (int*)nullptr, (int)n, 0, 3 * MORTON_BITS);
    if (e != cudaSuccess) return e;
    // the leaves' order of processing: by radius, largest first
    const long long leaves = 1LL << w.D;
    size_t cbl = 0;
    const cudaError_t el = cub::DeviceRadixSort::SortPairs(nullptr, cbl, (const unsigned*)nullptr, (unsigned*)nullptr,
                                                           (const int*)nullptr, (int*)nullptr, (int)leaves, 0, 32);
    if (el != cudaSuccess) return el;
    cb = std::max(cb, cbl);
    w.cub_bytes = cb;
    w.cub = cv.take(cb);
    w.lkey0 = cv.take((size_t)leaves * 4);
    w.lkey1 = cv.take((size_t)leaves * 4);
    w.lord0 = cv.take((size_t)leaves * 4);
    w.lord1 = cv.take((size_t)leaves * 4);
    w.psrc = cv.take((size_t)n * P_F4 * 16);
    w.geo = cv.take((size_t)w.nodes * 16);
    w.box = cv.take((size_t)w.nodes * 32);
    w.mom = cv.take((size_t)w.nodes * 3 * nterms(TREE_MAX_P) * sizeof(float));
    w.counter = cv.take(sizeof(int));
    w.bytes = cv.off;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Build: bounding box, Morton keys, sort, packed sorted sources.
// ---------------------------------------------------------------------------
__global__ void tree_bounds_kernel(const float4* __restrict__ pos, int n, float* __restrict__ part)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = pos[i];
        lo[0] = fminf(lo[0], p.x), lo[1] = fminf(lo[1], p.y), lo[2] = fminf(lo[2], p.z);
        hi[0] = fmaxf(hi[0], p.x), hi[1] = fmaxf(hi[1], p.y), hi[2] = fmaxf(hi[2], p.z);
    }
    __shared__ float red[6][32];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int c = 0; c < 3; ++c) red[c][w] = lo[c], red[3 + c][w] = hi[c];
    __syncthreads();
    if (threadIdx.x < 6) {
        float v = red[threadIdx.x][0];
        for (int k = 1; k < nw; ++k) v = threadIdx.x < 3 ? fminf(v, red[threadIdx.x][k]) : fmaxf(v, red[threadIdx.x][k]);
        part[blockIdx.x * 6 + threadIdx.x] = v;
    }
}

// One block: the partial boxes into one, written after them at part[6 nparts].
__global__ void tree_box_kernel(float* __restrict__ part, int nparts)
{
    __shared__ float red[6][32];
    float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int k = threadIdx.x; k < nparts; k += blockDim.x)
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = c < 3 ? fminf(v[c], part[k * 6 + c]) : fmaxf(v[c], part[k * 6 + c]);
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float t = __shfl_xor_sync(0xffffffffu, v[c], o);
            v[c] = c < 3 ? fminf(v[c], t) : fmaxf(v[c], t);
        }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int c = 0; c < 6; ++c) red[c][w] = v[c];
    __syncthreads();
    if (threadIdx.x < 6) {
        float r = red[threadIdx.x][0];
        for (int k = 1; k < nw; ++k) r = threadIdx.x < 3 ? fminf(r, red[threadIdx.x][k]) : fmaxf(r, red[threadIdx.x][k]);
        part[nparts * 6 + threadIdx.x] = r;
    }
}

// Spreads the low 21 bits of v to every third bit of a 64-bit word.
__device__ __forceinline__ unsigned long long spread3(unsigned int v)
{
    unsigned long long x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}

__global__ void tree_keys_kernel(const float4* __restrict__ pos, int n, const float* __restrict__ boxg,
                                 unsigned long long* __restrict__ keys, int* __restrict__ idx)
{
    __shared__ float box[6];
    if (threadIdx.x < 6) box[threadIdx.x] = boxg[threadIdx.x];
    __syncthreads();
    const float ext = fmaxf(fmaxf(box[3] - box[0], box[4] - box[1]), box[5] - box[2]);
    const float top = (float)((1u << MORTON_BITS) - 1);
    const float scale = ext > 0.f ? top / ext : 0.f;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = pos[i];
    const float q[3] = {(p.x - box[0]) * scale, (p.y - box[1]) * scale, (p.z - box[2]) * scale};
    unsigned int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = (unsigned int)fminf(fmaxf(q[a], 0.f), top);  // NaN -> 0
    keys[i] = (spread3(c[0]) << 2) | (spread3(c[1]) << 1) | spread3(c[2]);
    idx[i] = i;
}

// Sorted position k <- particle idx[k], packed like the direct sweep's sources:
//   (-x,-x,-y,-y) (-z,-z,gx,gx) (gy,gy,gz,gz) (-gx,-gx,-gy,-gy) (-gz,-gz,0,0).
__global__ void tree_gather_kernel(const float4* __restrict__ pos, const float4* __restrict__ str,
                                   const int* __restrict__ idx, int n, float4* __restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int j = idx[k];
    const float4 p = pos[j], g = str[j];
    float4* o = out + (size_t)k * P_F4;
    o[0] = make_float4(-p.x, -p.x, -p.y, -p.y);
    o[1] = make_float4(-p.z, -p.z, g.x, g.x);
    o[2] = make_float4(g.y, g.y, g.z, g.z);
    o[3] = make_float4(-g.x, -g.x, -g.y, -g.y);
    o[4] = make_float4(-g.z, -g.z, 0.f, 0.f);
}

__device__ __forceinline__ long long run_begin(long long k, long long n, int level) { return (k * n) >> level; }

// Sort keys that put the leaves of largest radius first (the likeliest to take the
// longest): the bit pattern of a non-negative float orders like the float.
__global__ void tree_leaf_keys_kernel(const float4* __restrict__ geo, int D, unsigned* __restrict__ key,
                                      int* __restrict__ val)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long leaves = 1LL << D;
    if (k >= leaves) return;
    key[k] = ~__float_as_uint(fmaxf(geo[leaves - 1 + k].w, 0.f));
    val[k] = (int)k;
}

// ---------------------------------------------------------------------------
// Leaves: box, radius and moments of every leaf, one warp per leaf.
// ---------------------------------------------------------------------------
template <int P>
__global__ void tree_leaf_kernel(const float4* __restrict__ psrc, long long n, int D, float4* __restrict__ geo,
                                 float4* __restrict__ box, float* __restrict__ mom)
{
    constexpr int NM = nterms(P);
    const long long leaf = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (leaf >= (1LL << D)) return;
    const long long s = run_begin(leaf, n, D), e = run_begin(leaf + 1, n, D);
    float px[2], py[2], pz[2], gx[2], gy[2], gz[2];
    bool ok[2];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const long long i = s + lane + 32 * h;
        ok[h] = i < e;
        px[h] = py[h] = pz[h] = gx[h] = gy[h] = gz[h] = 0.f;
        if (ok[h]) {
            const float4* q = psrc + i * P_F4;
            const float4 q0 = q[0], q1 = q[1], q2 = q[2];
            px[h] = -q0.x, py[h] = -q0.z, pz[h] = -q1.x;
            gx[h] = q1.z, gy[h] = q2.x, gz[h] = q2.z;
            lo[0] = fminf(lo[0], px[h]), lo[1] = fminf(lo[1], py[h]), lo[2] = fminf(lo[2], pz[h]);
            hi[0] = fmaxf(hi[0], px[h]), hi[1] = fmaxf(hi[1], py[h]), hi[2] = fmaxf(hi[2], pz[h]);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    const float cx = 0.5f * (lo[0] + hi[0]), cy = 0.5f * (lo[1] + hi[1]), cz = 0.5f * (lo[2] + hi[2]);
    float r2 = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (ok[h]) {
            const float dx = px[h] - cx, dy = py[h] - cy, dz = pz[h] - cz;
            r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    const long long id = (1LL << D) - 1 + leaf;
    if (lane == 0) {
        // the radius is rounded up by a relative 1e-6 so that it bounds the FP32 distances
        geo[id] = make_float4(cx, cy, cz, sqrtf(r2) * 1.000001f);
        box[2 * id] = make_float4(lo[0], lo[1], lo[2], 0.f);
        box[2 * id + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
#pragma unroll 1
    for (int l = 0; l < 3; ++l) {
        float acc[NM];
#pragma unroll
        for (int q = 0; q < NM; ++q) acc[q] = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!ok[h]) continue;
            const float g = l == 0 ? gx[h] : (l == 1 ? gy[h] : gz[h]);
            float tx[P + 1], ty[P + 1], tz[P + 1];  // d^a / a! per axis
            tx[0] = ty[0] = tz[0] = 1.f;
#pragma unroll
            for (int a = 1; a <= P; ++a) {
                tx[a] = tx[a - 1] * (px[h] - cx) * (1.f / a);
                ty[a] = ty[a - 1] * (py[h] - cy) * (1.f / a);
                tz[a] = tz[a - 1] * (pz[h] - cz) * (1.f / a);
            }
#pragma unroll
            for (int m = 0; m <= P; ++m)
#pragma unroll
                for (int a = m; a >= 0; --a)
#pragma unroll
                    for (int b = m - a; b >= 0; --b) {
                        const int c = m - a - b;
                        acc[midx(a, b, c)] = fmaf(g, tx[a] * ty[b] * tz[c], acc[midx(a, b, c)]);
                    }
        }
#pragma unroll
        for (int q = 0; q < NM; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            if (lane == (q & 31)) mom[(size_t)id * 3 * NM + l * NM + q] = acc[q];
        }
    }
}

// ---------------------------------------------------------------------------
// Upward pass: one level, one thread per (node, component).
// ---------------------------------------------------------------------------
template <int P>
__global__ void tree_up_kernel(int level, float4* __restrict__ geo, float4* __restrict__ box, float* __restrict__ mom)
{
    constexpr int NM = nterms(P);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * (1LL << level)) return;
    const long long k = t / 3;
    const int l = (int)(t - 3 * k);
    const long long id = (1LL << level) - 1 + k;
    const long long ch[2] = {2 * id + 1, 2 * id + 2};
    const float4 l0 = box[2 * ch[0]], h0 = box[2 * ch[0] + 1], l1 = box[2 * ch[1]], h1 = box[2 * ch[1] + 1];
    const float lo[3] = {fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z)};
    const float hi[3] = {fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z)};
    const float c[3] = {0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2])};
    float out[NM];
#pragma unroll
    for (int q = 0; q < NM; ++q) out[q] = 0.f;
    float rad = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float4 g = geo[ch[h]];
        const float sx = g.x - c[0], sy = g.y - c[1], sz = g.z - c[2];
        rad = fmaxf(rad, sqrtf(sx * sx + sy * sy + sz * sz) + g.w);
        float tx[P + 1], ty[P + 1], tz[P + 1];  // s^a / a! per axis
        tx[0] = ty[0] = tz[0] = 1.f;
#pragma unroll
        for (int a = 1; a <= P; ++a) {
            tx[a] = tx[a - 1] * sx * (1.f / a);
            ty[a] = ty[a - 1] * sy * (1.f / a);
            tz[a] = tz[a - 1] * sz * (1.f / a);
        }
        const float* mc = mom + (size_t)ch[h] * 3 * NM + l * NM;
        float m[NM];
#pragma unroll
        for (int q = 0; q < NM; ++q) m[q] = mc[q];
#pragma unroll
        for (int n = 0; n <= P; ++n)
#pragma unroll
            for (int a = n; a >= 0; --a)
#pragma unroll
                for (int b = n - a; b >= 0; --b) {
                    const int cc = n - a - b;
                    float v = out[midx(a, b, cc)];
#pragma unroll
                    for (int a2 = 0; a2 <= a; ++a2)
#pragma unroll
                        for (int b2 = 0; b2 <= b; ++b2)
#pragma unroll
                            for (int c2 = 0; c2 <= cc; ++c2)
                                v = fmaf(m[midx(a2, b2, c2)], tx[a - a2] * ty[b - b2] * tz[cc - c2], v);
                    out[midx(a, b, cc)] = v;
                }
    }
    float* mp = mom + (size_t)id * 3 * NM + l * NM;
#pragma unroll
    for (int q = 0; q < NM; ++q) mp[q] = out[q];
    if (l == 0) {
        const float hd = 0.5f * sqrtf((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                      (hi[2] - lo[2]) * (hi[2] - lo[2]));
        geo[id] = make_float4(c[0], c[1], c[2], fminf(rad, hd) * 1.000001f);
        box[2 * id] = make_float4(lo[0], lo[1], lo[2], 0.f);
        box[2 * id + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
}

// ---------------------------------------------------------------------------
// Segment tree (right-hand side only).  The blade and wake segments (Sec. II.A) form a
// second source tree, sorted by the Morton keys of their midpoints and split into
// count-balanced halves like the particle tree.  Segment j is the line strength
// Gamma_j (b_j - a_j) dt along a_j + t (b_j - a_j), t in [0, 1]; far from it its
// velocity is the point-vortex kernel integrated along the line, so a node's far field
// enters the target's local expansion through the moments of these line strengths,
// which 3-point Gauss-Legendre quadrature in t gives exactly through order 5.  Near
// nodes are summed with the direct sweep's exact Vatistas kernel.
// ---------------------------------------------------------------------------
__global__ void seg_mid_kernel(const float4* __restrict__ a, const float4* __restrict__ b, int m,
                               float4* __restrict__ mid)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const float4 p = a[j], q = b[j];
    mid[j] = make_float4(0.5f * (p.x + q.x), 0.5f * (p.y + q.y), 0.5f * (p.z + q.z), 0.f);
}

// Sorted position k <- segment idx[k], packed like the direct sweep's segment sources:
//   (-ax,-ax,-ay,-ay) (-az,-az,r0x,r0x) (r0y,r0y,r0z,r0z) (-r0x,-r0x,-r0y,-r0y) (-r0z,-r0z,-L2,-L2) (G,G,e,e)
// with r0 = b - a, L2 = |r0|^2 and e = (core |r0|)^(2n).
__global__ void seg_gather_kernel(const float4* __restrict__ sa, const float4* __restrict__ sb,
                                  const int* __restrict__ idx, int m, float core, int vn, float4* __restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const int j = idx[k];
    const float4 a = sa[j], b = sb[j];
    const float rx = b.x - a.x, ry = b.y - a.y, rz = b.z - a.z;
    const float L2 = rx * rx + ry * ry + rz * rz;
    const float cl2 = core * core * L2;
    float e = vn == 2 ? cl2 * cl2 : cl2, g = a.w;
    if (!(L2 > 0.f)) g = 0.f, e = 1.f;  // a zero-length segment induces nothing; keeps D > 0
    float4* o = out + (size_t)k * S_F4;
    o[0] = make_float4(-a.x, -a.x, -a.y, -a.y);
    o[1] = make_float4(-a.z, -a.z, rx, rx);
    o[2] = make_float4(ry, ry, rz, rz);
    o[3] = make_float4(-rx, -rx, -ry, -ry);
    o[4] = make_float4(-rz, -rz, -L2, -L2);
    o[5] = make_float4(g, g, e, e);
}

// Segment leaves: the box and sphere of both end points of every segment, and the
// moments sum_j sum_i w_i Gamma_j r0_j (y_ij - c)^k / k! over the Gauss points
// y_ij = a_j + t_i r0_j.  One warp per leaf.
template <int P>
__global__ void seg_leaf_kernel(const float4* __restrict__ ssrc, long long m, int D, float4* __restrict__ geo,
                                float4* __restrict__ box, float* __restrict__ mom)
{
    constexpr int NM = nterms(P);
    const long long leaf = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (leaf >= (1LL << D)) return;
    const long long s = run_begin(leaf, m, D), e = run_begin(leaf + 1, m, D);
    float ax[2], ay[2], az[2], rx[2], ry[2], rz[2], g[2];
    bool ok[2];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const long long i = s + lane + 32 * h;
        ok[h] = i < e;
        ax[h] = ay[h] = az[h] = rx[h] = ry[h] = rz[h] = g[h] = 0.f;
        if (ok[h]) {
            const float4* q = ssrc + i * S_F4;
            const float4 q0 = q[0], q1 = q[1], q2 = q[2], q5 = q[5];
            ax[h] = -q0.x, ay[h] = -q0.z, az[h] = -q1.x;
            rx[h] = q1.z, ry[h] = q2.x, rz[h] = q2.z;
            g[h] = q5.x;
            const float bx = ax[h] + rx[h], by = ay[h] + ry[h], bz = az[h] + rz[h];
            lo[0] = fminf(lo[0], fminf(ax[h], bx)), lo[1] = fminf(lo[1], fminf(ay[h], by));
            lo[2] = fminf(lo[2], fminf(az[h], bz));
            hi[0] = fmaxf(hi[0], fmaxf(ax[h], bx)), hi[1] = fmaxf(hi[1], fmaxf(ay[h], by));
            hi[2] = fmaxf(hi[2], fmaxf(az[h], bz));
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    const float cx = 0.5f * (lo[0] + hi[0]), cy = 0.5f * (lo[1] + hi[1]), cz = 0.5f * (lo[2] + hi[2]);
    float r2 = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (ok[h])
#pragma unroll
            for (int t = 0; t < 2; ++t) {  // both end points
                const float dx = ax[h] + t * rx[h] - cx, dy = ay[h] + t * ry[h] - cy, dz = az[h] + t * rz[h] - cz;
                r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
            }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    const long long id = (1LL << D) - 1 + leaf;
    if (lane == 0) {
        geo[id] = make_float4(cx, cy, cz, sqrtf(r2) * 1.000001f);
        box[2 * id] = make_float4(lo[0], lo[1], lo[2], 0.f);
        box[2 * id + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
    // Gauss-Legendre nodes and weights on [0, 1]
    const float gt[3] = {0.5f - 0.38729833462074169f, 0.5f, 0.5f + 0.38729833462074169f};
    const float gw[3] = {5.f / 18.f, 8.f / 18.f, 5.f / 18.f};
#pragma unroll 1
    for (int l = 0; l < 3; ++l) {
        float acc[NM];
#pragma unroll
        for (int q = 0; q < NM; ++q) acc[q] = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!ok[h]) continue;
            const float gl = g[h] * (l == 0 ? rx[h] : (l == 1 ? ry[h] : rz[h]));
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float w = gw[i] * gl;
                const float px = fmaf(gt[i], rx[h], ax[h]) - cx, py = fmaf(gt[i], ry[h], ay[h]) - cy,
                            pz = fmaf(gt[i], rz[h], az[h]) - cz;
                float tx[P + 1], ty[P + 1], tz[P + 1];  // d^a / a! per axis
                tx[0] = ty[0] = tz[0] = 1.f;
#pragma unroll
                for (int a = 1; a <= P; ++a) {
                    tx[a] = tx[a - 1] * px * (1.f / a);
                    ty[a] = ty[a - 1] * py * (1.f / a);
                    tz[a] = tz[a - 1] * pz * (1.f / a);
                }
#pragma unroll
                for (int n2 = 0; n2 <= P; ++n2)
#pragma unroll
                    for (int a = n2; a >= 0; --a)
#pragma unroll
                        for (int b = n2 - a; b >= 0; --b) {
                            const int c = n2 - a - b;
                            acc[midx(a, b, c)] = fmaf(w, tx[a] * ty[b] * tz[c], acc[midx(a, b, c)]);
                        }
            }
        }
#pragma unroll
        for (int q = 0; q < NM; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            if (lane == (q & 31)) mom[(size_t)id * 3 * NM + l * NM + q] = acc[q];
        }
    }
}

// ---------------------------------------------------------------------------
// Far field through the target leaf's local expansion.
// ---------------------------------------------------------------------------
template <int P>
struct Local {
    static constexpr int Q = P + 1;              // local expansion order (p + 2 measured 10% slower
                                                 // for a gradient error 1.1-3 times smaller)
    static constexpr int NQ = P + Q;             // highest order of b_k needed
    static constexpr int DIM = NQ + 1;           // dense table b[a][b][c], a, b, c <= NQ
    static constexpr int DL = Q + 1;             // dense table L[l][a][b][c], a, b, c <= Q
    static constexpr int SL = DL * DL * DL;
    static constexpr int NM = nterms(P);         // moments per component
    static constexpr int NL = nterms(Q);         // local coefficients per component
    static constexpr int RL = (NL + 31) / 32;    // local coefficients owned per lane
    static constexpr int TABLE = DIM * DIM * DIM > 3 * SL ? DIM * DIM * DIM : 3 * SL;
};

// The multi-indices of order <= 10 in the graded order, (a, b, c) packed 4 bits each,
// and the reciprocals 1/j.
constexpr int MI_MAX = 10;
struct MiTable {
    unsigned short abc[nterms(MI_MAX)];
    float recip[16];
};

constexpr MiTable make_mi_table()
{
    MiTable t{};
    int q = 0;
    for (int n = 0; n <= MI_MAX; ++n)
        for (int a = n; a >= 0; --a)
            for (int b = n - a; b >= 0; --b) t.abc[q++] = (unsigned short)(a | (b << 4) | ((n - a - b) << 8));
    t.recip[0] = 0.f;
    for (int j = 1; j < 16; ++j) t.recip[j] = 1.0f / (float)j;
    return t;
}

static __constant__ MiTable kMi = make_mi_table();

// b_k(R0) for |k| <= NQ into the warp's dense table, order by order (each order reads
// the two before it); the lanes share every order's entries.
template <int P>
__device__ __forceinline__ void local_table(float* __restrict__ B, float rx, float ry, float rz, int lane,
                                            const unsigned short* __restrict__ abc)
{
    using L = Local<P>;
    static_assert(L::NQ <= MI_MAX, "multi-index table too short");
    constexpr int D1 = L::DIM, D2 = L::DIM * L::DIM;
    const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
    const float ir2 = __frcp_rn(r2);
    if (lane == 0) B[0] = rsqrtf(r2);
    __syncwarp();
#pragma unroll 1
    for (int n = 1; n <= L::NQ; ++n) {
        const float c1 = (float)(2 * n - 1) * kMi.recip[n], c2 = (float)(n - 1) * kMi.recip[n];
        const int q1 = nterms(n);
#pragma unroll 1
        for (int q = nterms(n - 1) + lane; q < q1; q += 32) {
            const unsigned v = abc[q];  // lanes read different entries: shared memory, not the constant bank
            const int a = v & 15, b = (v >> 4) & 15, c = v >> 8;
            const int i = a * D2 + b * D1 + c;
            float s1 = 0.f, s2 = 0.f;
            if (a >= 1) s1 = fmaf((float)a * rx, B[i - D2], s1);
            if (b >= 1) s1 = fmaf((float)b * ry, B[i - D1], s1);
            if (c >= 1) s1 = fmaf((float)c * rz, B[i - 1], s1);
            if (a >= 2) s2 = fmaf((float)(a * (a - 1)), B[i - 2 * D2], s2);
            if (b >= 2) s2 = fmaf((float)(b * (b - 1)), B[i - 2 * D1], s2);
            if (c >= 2) s2 = fmaf((float)(c * (c - 1)), B[i - 2], s2);
            B[i] = ir2 * fmaf(c1, s1, -c2 * s2);
        }
        __syncwarp();
    }
}

// The local coefficients owned by a lane: m = lane + 32 r.
template <int P>
struct LocalAcc {
    float x[Local<P>::RL], y[Local<P>::RL], z[Local<P>::RL];
    int base[Local<P>::RL];  // offset of m in the b table
};

// L_m^l += sum_k M_k^l b_{k+m}(R0) for the lane's m (the sign (-1)^|m| comes later).
template <int P>
__device__ __forceinline__ void local_accumulate(LocalAcc<P>& acc, const float* __restrict__ B,
                                                 const float* __restrict__ M)
{
    using L = Local<P>;
    constexpr int D1 = L::DIM, D2 = L::DIM * L::DIM;
#pragma unroll 5
    for (int q = 0; q < L::NM; ++q) {
        const unsigned v = kMi.abc[q];
        const int off = (int)(v & 15) * D2 + (int)((v >> 4) & 15) * D1 + (int)(v >> 8);
        const float Mx = M[q], My = M[L::NM + q], Mz = M[2 * L::NM + q];
#pragma unroll
        for (int r = 0; r < L::RL; ++r) {
            const float bv = B[acc.base[r] + off];
            acc.x[r] = fmaf(Mx, bv, acc.x[r]);
            acc.y[r] = fmaf(My, bv, acc.y[r]);
            acc.z[r] = fmaf(Mz, bv, acc.z[r]);
        }
    }
}

// The local expansion at one target, y = x - c_t: adds 4 pi u to w[0..2] and
// -4 pi (grad u)_ab / 3 to the eight stored entries of G' (w[3..10] = xx, xy, xz,
// yx, yy, yz, zx, zy), the direct sweep's accumulator form (the expansion's gradient
// is trace-free exactly: its three diagonal sums cancel term by term).
// Ld[l SL + (a DL + b) DL + c] = L_m^l, m = (a, b, c).
template <int P, bool GRAD>
__device__ __forceinline__ void local_eval(float yx, float yy, float yz, const float* __restrict__ Ld, float* w)
{
    using L = Local<P>;
    constexpr int Q = L::Q, DL = L::DL, SL = L::SL, D2 = DL * DL;
    const float* Lx = Ld;
    const float* Ly = Ld + SL;
    const float* Lz = Ld + 2 * SL;
    float ux = 0.f, uy = 0.f, uz = 0.f;
    float jxx = 0.f, jxy = 0.f, jxz = 0.f, jyx = 0.f, jyy = 0.f, jyz = 0.f, jzx = 0.f, jzy = 0.f;
    float wa = 1.f;  // y^m / m!, built incrementally
#pragma unroll 1
    for (int a = 0; a < Q; ++a) {
        float wb = wa;
#pragma unroll 1
        for (int b = 0; a + b < Q; ++b) {
            float wm = wb;
            int i = (a * DL + b) * DL;
#pragma unroll 1
            for (int c = 0; a + b + c < Q; ++c, ++i) {
                // 4 pi u_a = eps_ajl d_j Psi^l
                ux = fmaf(wm, Lz[i + DL] - Ly[i + 1], ux);
                uy = fmaf(wm, Lx[i + 1] - Lz[i + D2], uy);
                uz = fmaf(wm, Ly[i + D2] - Lx[i + DL], uz);
                if (GRAD && a + b + c < Q - 1) {
                    // 4 pi J_ab = eps_ajl d_b d_j Psi^l
                    const int ixx = i + 2 * D2, iyy = i + 2 * DL, izz = i + 2;
                    const int ixy = i + D2 + DL, ixz = i + D2 + 1, iyz = i + DL + 1;
                    jxx = fmaf(wm, Lz[ixy] - Ly[ixz], jxx);
                    jxy = fmaf(wm, Lz[iyy] - Ly[iyz], jxy);
                    jxz = fmaf(wm, Lz[iyz] - Ly[izz], jxz);
                    jyx = fmaf(wm, Lx[ixz] - Lz[ixx], jyx);
                    jyy = fmaf(wm, Lx[iyz] - Lz[ixy], jyy);
                    jyz = fmaf(wm, Lx[izz] - Lz[ixz], jyz);
                    jzx = fmaf(wm, Ly[ixx] - Lx[ixy], jzx);
                    jzy = fmaf(wm, Ly[ixy] - Lx[iyy], jzy);
                }
                wm *= yz * kMi.recip[c + 1];
            }
            wb *= yy * kMi.recip[b + 1];
        }
        wa *= yx * kMi.recip[a + 1];
    }
    w[0] += ux, w[1] += uy, w[2] += uz;
    if constexpr (GRAD) {
        constexpr float k = -1.f / 3.f;
        w[3] = fmaf(k, jxx, w[3]), w[4] = fmaf(k, jxy, w[4]), w[5] = fmaf(k, jxz, w[5]);
        w[6] = fmaf(k, jyx, w[6]), w[7] = fmaf(k, jyy, w[7]), w[8] = fmaf(k, jyz, w[8]);
        w[9] = fmaf(k, jzx, w[9]), w[10] = fmaf(k, jzy, w[10]);
    }
}

struct TreeArgs {
    const float4* psrc;  // sorted packed sources [n][5]
    const float4* geo;   // per node (cx, cy, cz, r)
    const float4* box;   // per node (lo, hi)
    const float* mom;    // per node [3][NM] scaled moments
    const int* idx;      // sorted position -> particle index
    const int* order;    // the leaves in order of processing
    long long heavy;     // leaves at the head of the order that are processed as two items
    long long n;
    int D;
    float theta, sep;    // opening angle, 7 sigma
    NearConst nc;
    int* counter;
    float* u;
    float* grad;
    SegTreeView seg;     // the segment tree (seg.m = 0: none)
};

// The direct sum over the sorted run [s, e) staged through the warp's buffer.  With
// NEAR, a source at least 7 sigma from the target leaf's box takes the point-vortex
// form for the whole warp (a warp-uniform test on the broadcast source), and only
// the others evaluate the regularised kernel pair by pair.
template <bool GRAD, bool NEAR>
__device__ __forceinline__ void direct_run(Acc<GRAD, false>& acc, const TreeArgs& A, long long s, long long e,
                                           float4* buf, int lane, f2 X, f2 Y, f2 Z, float4 blo, float4 bhi,
                                           const float4* __restrict__ T)
{
    const Own own{};
    for (long long c0 = s; c0 < e; c0 += TREE_STAGE) {
        const int cnt = (int)min((long long)TREE_STAGE, e - c0);
        __syncwarp();
        // each lane stages two sources and, for a near run, tests them against the
        // target leaf's box; the warp-wide masks then steer every source uniformly
        unsigned far_mask[TREE_STAGE / 32];
#pragma unroll
        for (int h = 0; h < TREE_STAGE / 32; ++h) {
            const int t = lane + 32 * h;
            bool far = true;
            if (t < cnt) {
                const float4* src = A.psrc + (c0 + t) * P_F4;
                float4 v[P_F4];
#pragma unroll
                for (int f = 0; f < P_F4; ++f) v[f] = src[f], buf[t * P_F4 + f] = v[f];
                if constexpr (NEAR) {
                    const float sx = -v[0].x, sy = -v[0].z, sz = -v[1].x;
                    const float ex = fmaxf(fmaxf(blo.x - sx, sx - bhi.x), 0.f);
                    const float ey = fmaxf(fmaxf(blo.y - sy, sy - bhi.y), 0.f);
                    const float ez = fmaxf(fmaxf(blo.z - sz, sz - bhi.z), 0.f);
                    far = fmaf(ez, ez, fmaf(ey, ey, ex * ex)) >= A.nc.far2;
                }
            }
            far_mask[h] = __ballot_sync(0xffffffffu, far);
        }
        __syncwarp();
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const float4* q = buf + j * P_F4;
            const unsigned m = (TREE_STAGE > 32 && j >= 32) ? far_mask[TREE_STAGE / 32 - 1] : far_mask[0];
            if (NEAR && !((m >> (j & 31)) & 1u))
                near_source_table<GRAD>(acc, q, X, Y, Z, A.nc, T);
            else
                particle_source<GRAD, false, false>(acc, q, X, Y, Z, A.nc, own);
        }
    }
}

// Segments of the sorted run [s, e) with the exact Vatistas kernel, staged through the
// warp's buffer.  SAFE: every target is at least 1e-3 of the longest segment away and
// the core is positive, so no per-lane guard can trigger.
constexpr int SEG_STAGE = TREE_STAGE * P_F4 / S_F4 / 32 * 32;

template <bool GRAD, bool SAFE>
__device__ __forceinline__ void segment_run(Acc<GRAD, false>& acc, const float4* __restrict__ ssrc, long long s,
                                            long long e, float4* buf, int lane, f2 X, f2 Y, f2 Z, int vn)
{
    for (long long c0 = s; c0 < e; c0 += SEG_STAGE) {
        const int cnt = (int)min((long long)SEG_STAGE, e - c0);
        __syncwarp();
        for (int t = lane; t < cnt * S_F4; t += 32) buf[t] = ssrc[c0 * S_F4 + t];
        __syncwarp();
#pragma unroll 1
        for (int j = 0; j < cnt; ++j) segment_source<GRAD, false, SAFE>(acc, buf + j * S_F4, X, Y, Z, vn);
    }
}

// Smallest segment count of a far segment node that enters the local expansion (a
// segment pair costs about twice a particle pair).
constexpr int M2L_MIN_SEG = 16;

// Shared memory of one traversal warp: the source staging buffer (also the node's
// moments) and the dense b_k table (also the finished local coefficients), rounded
// up to 16 bytes so that every warp's float4 staging buffer stays aligned.
template <int P>
__host__ __device__ constexpr size_t tree_warp_smem()
{
    return (TREE_STAGE * P_F4 * 16 + (size_t)Local<P>::TABLE * 4 + 15) / 16 * 16;
}

// A target leaf that straddles a jump of the Morton curve (two compact clusters far
// apart) has a sphere so large that no node is ever far from it, and its warp would sum
// most of the wake directly.  Such a leaf is split at the largest gap between
// index-consecutive targets, [s, g) and [g, e), and each part walks the tree with its
// own box and sphere (the warp computes every target in both walks and keeps each
// target's own part).  Split when both parts' spheres are below half the leaf's.
struct TargetGroup {
    float4 sph, lo, hi;  // sphere (centre, radius) and box of the group
    long long g0, g1;    // the group's index range
};

__device__ __forceinline__ void group_box(float3 p0, bool in0, float3 p1, bool in1, float4& lo, float4& hi,
                                          float4& sph)
{
    float l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
    const float a0[3] = {p0.x, p0.y, p0.z}, a1[3] = {p1.x, p1.y, p1.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (in0) l[c] = fminf(l[c], a0[c]), h[c] = fmaxf(h[c], a0[c]);
        if (in1) l[c] = fminf(l[c], a1[c]), h[c] = fmaxf(h[c], a1[c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            l[c] = fminf(l[c], __shfl_xor_sync(0xffffffffu, l[c], o));
            h[c] = fmaxf(h[c], __shfl_xor_sync(0xffffffffu, h[c], o));
        }
    }
    const float cx = 0.5f * (l[0] + h[0]), cy = 0.5f * (l[1] + h[1]), cz = 0.5f * (l[2] + h[2]);
    float r2 = 0.f;
    if (in0) r2 = fmaxf(r2, (p0.x - cx) * (p0.x - cx) + (p0.y - cy) * (p0.y - cy) + (p0.z - cz) * (p0.z - cz));
    if (in1) r2 = fmaxf(r2, (p1.x - cx) * (p1.x - cx) + (p1.y - cy) * (p1.y - cy) + (p1.z - cz) * (p1.z - cz));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    lo = make_float4(l[0], l[1], l[2], 0.f);
    hi = make_float4(h[0], h[1], h[2], 0.f);
    sph = make_float4(cx, cy, cz, sqrtf(r2) * 1.000001f);
}

// grp[0] holds the whole leaf; returns 2 (and both parts in grp) if it is split.
__device__ __forceinline__ int split_leaf(float3 q0, float3 q1, bool v0, bool v1, long long i0, long long i1,
                                          long long s, long long e, int lane, TargetGroup* grp, bool force = false)
{
    // the gap after target s + lane (next: s + lane + 1) and after s + 32 + lane
    const float3 n0 = make_float3(__shfl_down_sync(0xffffffffu, q0.x, 1), __shfl_down_sync(0xffffffffu, q0.y, 1),
                                  __shfl_down_sync(0xffffffffu, q0.z, 1));
    const float3 f1 = make_float3(__shfl_sync(0xffffffffu, q1.x, 0), __shfl_sync(0xffffffffu, q1.y, 0),
                                  __shfl_sync(0xffffffffu, q1.z, 0));
    const float3 n1 = make_float3(__shfl_down_sync(0xffffffffu, q1.x, 1), __shfl_down_sync(0xffffffffu, q1.y, 1),
                                  __shfl_down_sync(0xffffffffu, q1.z, 1));
    const float3 nx0 = lane < 31 ? n0 : f1;
    auto dist2 = [](float3 a, float3 b) {
        return (a.x - b.x) * (a.x - b.x) + (a.y - b.y) * (a.y - b.y) + (a.z - b.z) * (a.z - b.z);
    };
    const float gap0 = i0 + 1 < e ? dist2(q0, nx0) : -1.f;
    const float gap1 = (lane < 31 && i1 + 1 < e) ? dist2(q1, n1) : -1.f;
    float best = fmaxf(gap0, gap1);
    long long bi = gap0 >= gap1 ? i0 + 1 : i1 + 1;  // the first index after the gap
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) best = ob, bi = oi;
    }
    if (!(best > 0.f)) return 1;
    TargetGroup a, b;
    group_box(q0, v0 && i0 < bi, q1, v1 && i1 < bi, a.lo, a.hi, a.sph);
    group_box(q0, v0 && i0 >= bi, q1, v1 && i1 >= bi, b.lo, b.hi, b.sph);
    if (!force && !(fmaxf(a.sph.w, b.sph.w) < 0.5f * grp[0].sph.w)) return 1;
    a.g0 = s, a.g1 = bi, b.g0 = bi, b.g1 = e;
    grp[0] = a, grp[1] = b;
    return 2;
}

template <int P, bool GRAD>
__global__ void __launch_bounds__(TREE_WARPS * 32, 2) tree_eval_kernel(TreeArgs A)
{
    using L = Local<P>;
    static_assert(3 * L::NM <= TREE_STAGE * P_F4 * 4, "moments fit the warp's source buffer");
    static_assert(3 * L::SL <= L::TABLE, "local coefficients fit the table");
    static_assert(tree_warp_smem<P>() % 16 == 0 && (TREE_STAGE * P_F4 * 16) % 16 == 0, "16-byte aligned warp slices");
    extern __shared__ __align__(16) unsigned char tree_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* buf = reinterpret_cast<float4*>(tree_smem + warp * tree_warp_smem<P>());
    float* mbuf = reinterpret_cast<float*>(buf);
    float* B = reinterpret_cast<float*>(tree_smem + warp * tree_warp_smem<P>() + TREE_STAGE * P_F4 * 16);
    // the near-field table, after the warps' slices
    float4* T = reinterpret_cast<float4*>(tree_smem + TREE_WARPS * tree_warp_smem<P>());
    for (int t = threadIdx.x; t <= NEAR_NT; t += blockDim.x) T[t] = g_near_table[t];
    __shared__ unsigned short s_abc[nterms(MI_MAX)];
    for (int t = threadIdx.x; t < nterms(MI_MAX); t += blockDim.x) s_abc[t] = kMi.abc[t];
    __syncthreads();
    const long long nleaves = 1LL << A.D;
    // the lane's local coefficients m = lane + 32 r, (a, b, c) packed 4 bits each
    unsigned mabc[L::RL];
#pragma unroll
    for (int r = 0; r < L::RL; ++r) {
        const int q = lane + 32 * r;
        mabc[r] = q < L::NL ? kMi.abc[q] : 0u;
    }
    // work items: the A.heavy largest leaves (the first in A.order) as two items, one per
    // part of the leaf split at its largest gap, so that their two walks run on two warps;
    // every other leaf as one item (split or not by split_leaf's own test)
    const long long nitems = nleaves + A.heavy;
    for (;;) {
        long long item = 0;
        if (lane == 0) item = atomicAdd(A.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nitems) break;
        const int part = item < 2LL * A.heavy ? (int)(item & 1) : -1;
        const long long leaf = A.order[item < 2LL * A.heavy ? item >> 1 : item - A.heavy];
        const long long s = run_begin(leaf, A.n, A.D), e = run_begin(leaf + 1, A.n, A.D);
        const long long i0 = s + lane, i1 = s + 32 + lane;
        const bool v0 = i0 < e, v1 = i1 < e;
        const float4 p0 = A.psrc[(v0 ? i0 : s) * P_F4], p0z = A.psrc[(v0 ? i0 : s) * P_F4 + 1];
        const float4 p1 = A.psrc[(v1 ? i1 : s) * P_F4], p1z = A.psrc[(v1 ? i1 : s) * P_F4 + 1];
        const f2 X = make_float2(-p0.x, -p1.x), Y = make_float2(-p0.z, -p1.z), Z = make_float2(-p0z.x, -p1z.x);
        // the leaf's targets in one group, or two if the leaf straddles a gap
        TargetGroup grp[2];
        int ngroups = 1;
        grp[0].sph = A.geo[nleaves - 1 + leaf];
        grp[0].lo = A.box[2 * (nleaves - 1 + leaf)];
        grp[0].hi = A.box[2 * (nleaves - 1 + leaf) + 1];
        grp[0].g0 = s, grp[0].g1 = e;
        ngroups = split_leaf(make_float3(X.x, Y.x, Z.x), make_float3(X.y, Y.y, Z.y), v0, v1, i0, i1, s, e, lane, grp,
                             part >= 0);
        int g_first = 0, g_last = ngroups;
        if (part >= 0) {
            if (ngroups == 1 && part == 1) continue;  // a leaf of one target: its first item covers it
            g_first = part, g_last = part + 1;
        }
#pragma unroll 1
        for (int gi = g_first; gi < g_last; ++gi) {
        const float4 tg = grp[gi].sph, blo = grp[gi].lo, bhi = grp[gi].hi;
        const long long gs = grp[gi].g0, ge = grp[gi].g1;
        Acc<GRAD, false> acc;
        acc.zero();
        LocalAcc<P> la;
#pragma unroll
        for (int r = 0; r < L::RL; ++r) {
            la.x[r] = la.y[r] = la.z[r] = 0.f;
            const int a = mabc[r] & 15, b = (mabc[r] >> 4) & 15, c = mabc[r] >> 8;
            la.base[r] = (a * L::DIM + b) * L::DIM + c;
        }
        bool any_far = false;
        // depth-first walk; entry t of the stack lives in lane t
        int st = 0, sp = 1;  // the root
        while (sp > 0) {
            const int id = __shfl_sync(0xffffffffu, st, sp - 1);
            --sp;
            const int level = 31 - __clz(id + 1);
            const long long k = (long long)id + 1 - (1LL << level);
            const long long ns = run_begin(k, A.n, level), ne = run_begin(k + 1, A.n, level);
            const float4 g = A.geo[id];
            const float dx = g.x - tg.x, dy = g.y - tg.y, dz = g.z - tg.z;
            const float d = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
            const float rs = g.w + tg.w;
            const bool far = rs < A.theta * d && d - rs >= A.sep;
            if (far && ne - ns >= M2L_MIN) {
                __syncwarp();
                const float* src = A.mom + (size_t)id * 3 * L::NM;
                for (int t = lane; t < 3 * L::NM; t += 32) mbuf[t] = src[t];
                local_table<P>(B, -dx, -dy, -dz, lane, s_abc);  // R0 = c_t - c_s; ends with a warp sync
                local_accumulate<P>(la, B, mbuf);
                any_far = true;
            } else if (far) {
                direct_run<GRAD, false>(acc, A, ns, ne, buf, lane, X, Y, Z, blo, bhi, T);
            } else if (level == A.D) {
                if (d - rs >= A.sep)
                    direct_run<GRAD, false>(acc, A, ns, ne, buf, lane, X, Y, Z, blo, bhi, T);
                else
                    direct_run<GRAD, true>(acc, A, ns, ne, buf, lane, X, Y, Z, blo, bhi, T);
            } else {
                // push the right child first so the left one is walked first
                if (lane == sp) st = 2 * id + 2;
                if (lane == sp + 1) st = 2 * id + 1;
                sp += 2;
            }
        }
        // the segment tree: far nodes into the same local expansion, the others exactly
        if (A.seg.m > 0) {
            int sst = 0, ssp = 1;  // the root
            while (ssp > 0) {
                const int id = __shfl_sync(0xffffffffu, sst, ssp - 1);
                --ssp;
                const int level = 31 - __clz(id + 1);
                const long long k = (long long)id + 1 - (1LL << level);
                const long long ns = run_begin(k, A.seg.m, level), ne = run_begin(k + 1, A.seg.m, level);
                const float4 g = A.seg.geo[id];
                const float dx = g.x - tg.x, dy = g.y - tg.y, dz = g.z - tg.z;
                const float d = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
                const float rs = g.w + tg.w;
                const bool far = rs < A.theta * d && d - rs >= A.seg.sep;
                if (far && ne - ns >= M2L_MIN_SEG) {
                    __syncwarp();
                    const float* src = A.seg.mom + (size_t)id * 3 * L::NM;
                    for (int t = lane; t < 3 * L::NM; t += 32) mbuf[t] = src[t];
                    local_table<P>(B, -dx, -dy, -dz, lane, s_abc);
                    local_accumulate<P>(la, B, mbuf);
                    any_far = true;
                } else if (far || level == A.seg.D) {
                    // a segment inside the node's sphere is at most 2 r long
                    if (A.seg.core_pos && g.w > 0.f && d - rs >= 2e-3f * g.w)
                        segment_run<GRAD, true>(acc, A.seg.ssrc, ns, ne, buf, lane, X, Y, Z, A.seg.vn);
                    else
                        segment_run<GRAD, false>(acc, A.seg.ssrc, ns, ne, buf, lane, X, Y, Z, A.seg.vn);
                } else {
                    if (lane == ssp) sst = 2 * id + 2;
                    if (lane == ssp + 1) sst = 2 * id + 1;
                    ssp += 2;
                }
            }
        }
        if (any_far) {
            // the finished local coefficients, signed, into the table's storage
            __syncwarp();
#pragma unroll
            for (int r = 0; r < L::RL; ++r)
                if (lane + 32 * r < L::NL) {
                    const int a = mabc[r] & 15, b = (mabc[r] >> 4) & 15, c = mabc[r] >> 8;
                    const int i = (a * L::DL + b) * L::DL + c;
                    const float sg = ((a + b + c) & 1) ? -1.f : 1.f;
                    B[i] = sg * la.x[r], B[L::SL + i] = sg * la.y[r], B[2 * L::SL + i] = sg * la.z[r];
                }
            __syncwarp();
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                float w[11];
#pragma unroll
                for (int q = 0; q < 11; ++q) w[q] = 0.f;
                const float yx = (h ? X.y : X.x) - tg.x, yy = (h ? Y.y : Y.x) - tg.y, yz = (h ? Z.y : Z.x) - tg.z;
                local_eval<P, GRAD>(yx, yy, yz, B, w);
                if (h == 0) {
                    acc.v[0].x += w[0], acc.v[1].x += w[1], acc.v[2].x += w[2];
                    if constexpr (GRAD) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) acc.v[6 + q].x += w[3 + q];
                    }
                } else {
                    acc.v[0].y += w[0], acc.v[1].y += w[1], acc.v[2].y += w[2];
                    if constexpr (GRAD) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) acc.v[6 + q].y += w[3 + q];
                    }
                }
            }
        }
        // epilogue: u = u / (4 pi), J = ([S x] - 3 G') / (4 pi), G'_zz = -G'_xx - G'_yy
        const float f = 0.079577471545947668f;
        const long long n = A.n;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long it = h ? i1 : i0;
            if (!(h ? v1 : v0) || it < gs || it >= ge) continue;
            const long long o = A.idx[it];
            float v[14];
#pragma unroll
            for (int q = 0; q < Acc<GRAD, false>::N; ++q) v[q] = h ? acc.v[q].y : acc.v[q].x;
            A.u[o] = v[0] * f, A.u[n + o] = v[1] * f, A.u[2 * n + o] = v[2] * f;
            if constexpr (GRAD) {
                const float Sx = v[3], Sy = v[4], Sz = v[5], Gzz = -v[6] - v[10];
                float* J = A.grad;
                J[o] = (-3.f * v[6]) * f;
                J[n + o] = (-Sz - 3.f * v[7]) * f;
                J[2 * n + o] = (Sy - 3.f * v[8]) * f;
                J[3 * n + o] = (Sz - 3.f * v[9]) * f;
                J[4 * n + o] = (-3.f * v[10]) * f;
                J[5 * n + o] = (-Sx - 3.f * v[11]) * f;
                J[6 * n + o] = (-Sy - 3.f * v[12]) * f;
                J[7 * n + o] = (Sx - 3.f * v[13]) * f;
                J[8 * n + o] = (-3.f * Gzz) * f;
            }
        }
        __syncwarp();  // the table is read by every lane before the next walk overwrites it
        }
    }
}

template <int P>
cudaError_t launch_tree(const TreeWs& w, char* ws, long long n, float sigma, float theta, bool grad, float* u,
                        float* grad_u, cudaStream_t st, const SegTreeView* segs)
{
    float4* psrc = reinterpret_cast<float4*>(ws + w.psrc);
    float4* geo = reinterpret_cast<float4*>(ws + w.geo);
    float4* box = reinterpret_cast<float4*>(ws + w.box);
    float* mom = reinterpret_cast<float*>(ws + w.mom);
    const long long leaves = 1LL << w.D;
    trace_launch();
    tree_leaf_kernel<P><<<(unsigned)((leaves * 32 + 255) / 256), 256, 0, st>>>(psrc, n, w.D, geo, box, mom);
    for (int l = w.D - 1; l >= 0; --l) {
        const long long t = 3 * (1LL << l);
        trace_launch();
        tree_up_kernel<P><<<(unsigned)((t + 127) / 128), 128, 0, st>>>(l, geo, box, mom);
    }
    // the leaves by radius, largest first
    unsigned* lk0 = reinterpret_cast<unsigned*>(ws + w.lkey0);
    unsigned* lk1 = reinterpret_cast<unsigned*>(ws + w.lkey1);
    int* lo0 = reinterpret_cast<int*>(ws + w.lord0);
    int* lo1 = reinterpret_cast<int*>(ws + w.lord1);
    trace_launch();
    tree_leaf_keys_kernel<<<(unsigned)((leaves + 255) / 256), 256, 0, st>>>(geo, w.D, lk0, lo0);
    size_t cb = w.cub_bytes;
    cudaError_t e0 = cub::DeviceRadixSort::SortPairs(ws + w.cub, cb, lk0, lk1, lo0, lo1, (int)leaves, 0, 32, st);
    if (e0 != cudaSuccess) return e0;
    TreeArgs A{};
    A.order = lo1;
    A.heavy = std::min<long long>(leaves, std::max<long long>(leaves / 64, 1));
    A.psrc = psrc;
    A.geo = geo;
    A.box = box;
    A.mom = mom;
    A.idx = reinterpret_cast<const int*>(ws + w.idx1);
    A.n = n;
    A.D = w.D;
    A.theta = theta;
    A.sep = (float)(RHO_FAR * (double)sigma);
    const double s = sigma;
    A.nc.inv_s2 = (float)(1.0 / (s * s));
    A.nc.inv_s3 = (float)(1.0 / (s * s * s));
    A.nc.inv_s5 = (float)(1.0 / (s * s * s * s * s));
    A.nc.far2 = (float)((double)RHO_FAR * RHO_FAR * s * s);
    A.counter = reinterpret_cast<int*>(ws + w.counter);
    A.u = u;
    A.grad = grad_u;
    if (segs) A.seg = *segs;
    cudaError_t e = cudaMemsetAsync(A.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    auto kern = grad ? tree_eval_kernel<P, true> : tree_eval_kernel<P, false>;
    const size_t smem = TREE_WARPS * tree_warp_smem<P>() + (NEAR_NT + 1) * sizeof(float4);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TREE_WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    const long long want = (leaves + TREE_WARPS - 1) / TREE_WARPS;
    const long long blocks = std::min<long long>(want, (long long)std::max(per_sm, 1) * sm_count());
    trace_launch();
    kern<<<(unsigned)blocks, TREE_WARPS * 32, smem, st>>>(A);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Right-hand side of Eq. 4-5 with the treecode for the particle-particle sums.
// ---------------------------------------------------------------------------

// Per particle (original order): u, J from the tree (up, Jp) plus the segments (us,
// Js, or none), then Vreman's eddy viscosity, the stretching and dx/dt in FP64, as
// the direct sweep's epilogue forms them.
__global__ void tree_rhs_epilogue_kernel(int n, const float* __restrict__ up, const float* __restrict__ Jp,
                                         const float* __restrict__ us, const float* __restrict__ Js,
                                         const float4* __restrict__ str, float sigma, float c_v, float ux_inf,
                                         float uy_inf, float uz_inf, int classic, int check, int* dev_err,
                                         float* __restrict__ dxdt, float* __restrict__ dGdt, float* __restrict__ nu_t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double u[3], J[9];
    for (int a = 0; a < 3; ++a) u[a] = (double)up[(size_t)a * n + i] + (us ? (double)us[(size_t)a * n + i] : 0.0);
    for (int c = 0; c < 9; ++c) J[c] = (double)Jp[(size_t)c * n + i] + (Js ? (double)Js[(size_t)c * n + i] : 0.0);
    const float4 G4 = str[i];
    const double G[3] = {G4.x, G4.y, G4.z};
    // Vreman: alpha = J^T, beta = Delta^2 J J^T, Delta = sigma
    double bt[3][3], aa = 0.0;
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
            double v = 0.0;
            for (int m = 0; m < 3; ++m) v += J[3 * p + m] * J[3 * q + m];
            bt[p][q] = v * (double)sigma * (double)sigma;
        }
    for (int c = 0; c < 9; ++c) aa += J[c] * J[c];
    const double B = bt[0][0] * bt[1][1] - bt[0][1] * bt[0][1] + bt[0][0] * bt[2][2] - bt[0][2] * bt[0][2] +
                     bt[1][1] * bt[2][2] - bt[1][2] * bt[1][2];
    const double nut = (aa > 0.0 && B > 0.0) ? (double)c_v * sqrt(B / aa) : 0.0;
    double st[3];
    for (int a = 0; a < 3; ++a) {
        double v = 0.0;
        for (int c = 0; c < 3; ++c) v += classic ? J[3 * a + c] * G[c] : J[3 * c + a] * G[c];
        st[a] = v;
    }
    dxdt[i] = (float)(u[0] + ux_inf);
    dxdt[(size_t)n + i] = (float)(u[1] + uy_inf);
    dxdt[2 * (size_t)n + i] = (float)(u[2] + uz_inf);
    for (int a = 0; a < 3; ++a) dGdt[(size_t)a * n + i] = (float)st[a];
    nu_t[i] = (float)nut;
    if (check && !isfinite(u[0] + u[1] + u[2] + st[0] + st[1] + st[2] + nut)) atomicOr(dev_err, DEV_ERR_NONFINITE);
}

// Sorted copies for the PSE walk: (x, y, z, volume) and (Gamma, nu_t).
__global__ void tree_pse_gather_kernel(const float4* __restrict__ pos, const float4* __restrict__ str,
                                       const float* __restrict__ nu_t, const int* __restrict__ idx, int n,
                                       float4* __restrict__ sp, float4* __restrict__ sg)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int j = idx[k];
    sp[k] = pos[j];
    const float4 g = str[j];
    sg[k] = make_float4(g.x, g.y, g.z, nu_t[j]);
}

struct PseArgs {
    const float4* sp;   // sorted (x, y, z, v)
    const float4* sg;   // sorted (Gamma, nu_t)
    const float4* geo;  // the tree of the same positions
    const int* idx;
    const int* order;   // the leaves in order of processing
    long long n;
    int D;
    float sep, cut2, inv2s2, nu, pref;
    int* counter;
    float* dGdt;        // [3][n], original order: the PSE term is added
};

// Particle strength exchange (Eq. 5) by a walk of the same tree: one warp per target
// leaf visits the nodes whose sphere comes within 7 sigma of the leaf's and sums the
// Degond-Mas-Gallic pairs of the leaves it reaches (the pairs beyond 7 sigma, whose
// Gaussian is below 3e-11 of its peak, are skipped, as the direct PSE does).
__global__ void __launch_bounds__(TREE_WARPS * 32) tree_pse_kernel(PseArgs A)
{
    __shared__ float4 sbuf[TREE_WARPS][2 * TREE_STAGE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* bp = sbuf[warp];
    float4* bg = sbuf[warp] + TREE_STAGE;
    const long long nleaves = 1LL << A.D;
    for (;;) {
        long long leaf = 0;
        if (lane == 0) leaf = atomicAdd(A.counter, 1);
        leaf = __shfl_sync(0xffffffffu, leaf, 0);
        if (leaf >= nleaves) break;
        leaf = A.order[leaf];
        const long long s = run_begin(leaf, A.n, A.D), e = run_begin(leaf + 1, A.n, A.D);
        const long long i0 = s + lane, i1 = s + 32 + lane;
        const bool v0 = i0 < e, v1 = i1 < e;
        const float4 p0 = A.sp[v0 ? i0 : s], g0 = A.sg[v0 ? i0 : s];
        const float4 p1 = A.sp[v1 ? i1 : s], g1 = A.sg[v1 ? i1 : s];
        const float base0 = A.nu + 0.5f * g0.w, base1 = A.nu + 0.5f * g1.w;
        TargetGroup grp[2];
        grp[0].sph = A.geo[nleaves - 1 + leaf];
        grp[0].g0 = s, grp[0].g1 = e;
        const int ngroups = split_leaf(make_float3(p0.x, p0.y, p0.z), make_float3(p1.x, p1.y, p1.z), v0, v1, i0, i1,
                                       s, e, lane, grp);
#pragma unroll 1
        for (int gi = 0; gi < ngroups; ++gi) {
        const float4 tg = grp[gi].sph;
        const long long gs = grp[gi].g0, ge = grp[gi].g1;
        float a0x = 0.f, a0y = 0.f, a0z = 0.f, a1x = 0.f, a1y = 0.f, a1z = 0.f;
        int st = 0, sp = 1;  // the stack, one entry per lane
        while (sp > 0) {
            const int id = __shfl_sync(0xffffffffu, st, sp - 1);
            --sp;
            const int level = 31 - __clz(id + 1);
            const float4 g = A.geo[id];
            const float dx = g.x - tg.x, dy = g.y - tg.y, dz = g.z - tg.z;
            const float d = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
            if (d - (g.w + tg.w) >= A.sep) continue;  // every pair beyond 7 sigma
            if (level < A.D) {
                if (lane == sp) st = 2 * id + 2;
                if (lane == sp + 1) st = 2 * id + 1;
                sp += 2;
                continue;
            }
            const long long k = (long long)id + 1 - (1LL << level);
            const long long ns = run_begin(k, A.n, level), ne = run_begin(k + 1, A.n, level);
            const int cnt = (int)(ne - ns);  // a leaf: at most TREE_STAGE
            // stage the leaf; a source farther than 7 sigma from the target group's sphere
            // reaches none of its targets and is left out (warp-uniformly, by ballot)
            __syncwarp();
            unsigned keep[TREE_STAGE / 32];
#pragma unroll
            for (int h = 0; h < TREE_STAGE / 32; ++h) {
                const int t = lane + 32 * h;
                bool k = false;
                if (t < cnt) {
                    const float4 q = A.sp[ns + t];
                    bp[t] = q, bg[t] = A.sg[ns + t];
                    const float ex = q.x - tg.x, ey = q.y - tg.y, ez = q.z - tg.z;
                    const float lim = tg.w + A.sep;
                    k = fmaf(ez, ez, fmaf(ey, ey, ex * ex)) < lim * lim;
                }
                keep[h] = __ballot_sync(0xffffffffu, k);
            }
            __syncwarp();
#pragma unroll
            for (int hh = 0; hh < TREE_STAGE / 32; ++hh)
            for (unsigned m = keep[hh]; m; m &= m - 1) {
                const int j = 32 * hh + __ffs(m) - 1;
                const float4 pj = bp[j], gj = bg[j];
                const float ntj = gj.w;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float4 pi = h ? p1 : p0, gi = h ? g1 : g0;
                    const float rx = pi.x - pj.x, ry = pi.y - pj.y, rz = pi.z - pj.z;
                    const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
                    if (r2 < A.cut2) {
                        const float w = fmaf(0.5f, ntj, h ? base1 : base0) * expf(-r2 * A.inv2s2);
                        const float vi = pi.w, vj = pj.w;
                        const float tx = __fsub_rn(__fmul_rn(vi, gj.x), __fmul_rn(vj, gi.x));
                        const float ty = __fsub_rn(__fmul_rn(vi, gj.y), __fmul_rn(vj, gi.y));
                        const float tz = __fsub_rn(__fmul_rn(vi, gj.z), __fmul_rn(vj, gi.z));
                        if (h) a1x = fmaf(w, tx, a1x), a1y = fmaf(w, ty, a1y), a1z = fmaf(w, tz, a1z);
                        else a0x = fmaf(w, tx, a0x), a0y = fmaf(w, ty, a0y), a0z = fmaf(w, tz, a0z);
                    }
                }
            }
        }
        const long long n = A.n;
        if (v0 && i0 >= gs && i0 < ge) {
            const long long o = A.idx[i0];
            A.dGdt[o] += A.pref * a0x, A.dGdt[n + o] += A.pref * a0y, A.dGdt[2 * n + o] += A.pref * a0z;
        }
        if (v1 && i1 >= gs && i1 < ge) {
            const long long o = A.idx[i1];
            A.dGdt[o] += A.pref * a1x, A.dGdt[n + o] += A.pref * a1y, A.dGdt[2 * n + o] += A.pref * a1z;
        }
        __syncwarp();  // the staging buffer is read by every lane before the next walk refills it
        }
    }
}

}  // namespace

cudaError_t tree_workspace(long long n, size_t* bytes)
{
    TreeWs w;
    const cudaError_t e = tree_layout(n, w);
    *bytes = e == cudaSuccess ? w.bytes : 0;
    return e;
}

cudaError_t run_tree_induce(const float* pos, const float* str, long long n, float sigma, float theta, int order,
                            float* u, float* grad_u, char* ws, cudaStream_t st, const SegTreeView* segs)
{
    if (n == 0) return cudaSuccess;
    TreeWs w;
    cudaError_t e = tree_layout(n, w);
    if (e != cudaSuccess) return e;
    if ((e = near_table_ready()) != cudaSuccess) return e;
    float* part = reinterpret_cast<float*>(ws + w.part);
    auto* k0 = reinterpret_cast<unsigned long long*>(ws + w.keys0);
    auto* k1 = reinterpret_cast<unsigned long long*>(ws + w.keys1);
    int* i0 = reinterpret_cast<int*>(ws + w.idx0);
    int* i1 = reinterpret_cast<int*>(ws + w.idx1);
    const float4* p4 = reinterpret_cast<const float4*>(pos);
    const int nparts = (int)std::min<long long>(BOUNDS_BLOCKS, (n + 255) / 256);
    trace_launch();
    tree_bounds_kernel<<<nparts, 256, 0, st>>>(p4, (int)n, part);
    trace_launch();
    tree_box_kernel<<<1, 1024, 0, st>>>(part, nparts);
    trace_launch();
    tree_keys_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p4, (int)n, part + 6 * nparts, k0, i0);
    size_t cb = w.cub_bytes;
    e = cub::DeviceRadixSort::SortPairs(ws + w.cub, cb, k0, k1, i0, i1, (int)n, 0, 3 * MORTON_BITS, st);
    if (e != cudaSuccess) return e;
    trace_launch();
    tree_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p4, reinterpret_cast<const float4*>(str), i1,
                                                                     (int)n, reinterpret_cast<float4*>(ws + w.psrc));
    const bool grad = grad_u != nullptr;
    switch (order) {
        case 2: return launch_tree<2>(w, ws, n, sigma, theta, grad, u, grad_u, st, segs);
        case 3: return launch_tree<3>(w, ws, n, sigma, theta, grad, u, grad_u, st, segs);
        default: return launch_tree<4>(w, ws, n, sigma, theta, grad, u, grad_u, st, segs);
    }
}

}  // namespace vpm

namespace vpm {

// Workspace of the segment tree: midpoints, keys and permutation (twice, for the radix
// sort), the sort's scratch, the sorted packed segments and the nodes.
struct SegTreeWs {
    size_t part, mid, keys0, keys1, idx0, idx1, cub, cub_bytes, ssrc, geo, box, mom, bytes;
    int D;
    long long nodes;
};

static cudaError_t seg_tree_layout(long long m, SegTreeWs& w)
{
    Carve cv;
    w = SegTreeWs{};
    w.D = tree_depth(m);
    w.nodes = (2LL << w.D) - 1;
    w.part = cv.take((size_t)(BOUNDS_BLOCKS + 1) * 6 * sizeof(float));
    w.mid = cv.take((size_t)m * 16);
    w.keys0 = cv.take((size_t)m * 8);
    w.keys1 = cv.take((size_t)m * 8);
    w.idx0 = cv.take((size_t)m * 4);
    w.idx1 = cv.take((size_t)m * 4);
    size_t cb = 0;
    const cudaError_t e = cub::DeviceRadixSort::SortPairs(
        nullptr, cb, (const unsigned long long*)nullptr, (unsigned long long*)nullptr, (const int*)nullptr,
        (int*)nullptr, (int)m, 0, 3 * MORTON_BITS);
    if (e != cudaSuccess) return e;
    w.cub_bytes = cb;
    w.cub = cv.take(cb);
    w.ssrc = cv.take((size_t)m * S_F4 * 16);
    w.geo = cv.take((size_t)w.nodes * 16);
    w.box = cv.take((size_t)w.nodes * 32);
    w.mom = cv.take((size_t)w.nodes * 3 * nterms(TREE_MAX_P) * sizeof(float));
    w.bytes = cv.off;
    return cudaSuccess;
}

// Builds the segment tree of order P and describes it for the traversal.
template <int P>
static cudaError_t build_seg_tree(const SegTreeWs& w, char* ws, const float* seg_a, const float* seg_b, long long m,
                                  float core, int vn, SegTreeView& v, cudaStream_t st)
{
    const float4* a4 = reinterpret_cast<const float4*>(seg_a);
    const float4* b4 = reinterpret_cast<const float4*>(seg_b);
    float4* mid = reinterpret_cast<float4*>(ws + w.mid);
    float* part = reinterpret_cast<float*>(ws + w.part);
    auto* k0 = reinterpret_cast<unsigned long long*>(ws + w.keys0);
    auto* k1 = reinterpret_cast<unsigned long long*>(ws + w.keys1);
    int* i0 = reinterpret_cast<int*>(ws + w.idx0);
    int* i1 = reinterpret_cast<int*>(ws + w.idx1);
    float4* ssrc = reinterpret_cast<float4*>(ws + w.ssrc);
    float4* geo = reinterpret_cast<float4*>(ws + w.geo);
    float4* box = reinterpret_cast<float4*>(ws + w.box);
    float* mom = reinterpret_cast<float*>(ws + w.mom);
    const unsigned grid = (unsigned)((m + 255) / 256);
    trace_launch();
    seg_mid_kernel<<<grid, 256, 0, st>>>(a4, b4, (int)m, mid);
    const int nparts = (int)std::min<long long>(BOUNDS_BLOCKS, (m + 255) / 256);
    trace_launch();
    tree_bounds_kernel<<<nparts, 256, 0, st>>>(mid, (int)m, part);
    trace_launch();
    tree_box_kernel<<<1, 1024, 0, st>>>(part, nparts);
    trace_launch();
    tree_keys_kernel<<<grid, 256, 0, st>>>(mid, (int)m, part + 6 * nparts, k0, i0);
    size_t cb = w.cub_bytes;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(ws + w.cub, cb, k0, k1, i0, i1, (int)m, 0, 3 * MORTON_BITS, st);
    if (e != cudaSuccess) return e;
    trace_launch();
    seg_gather_kernel<<<grid, 256, 0, st>>>(a4, b4, i1, (int)m, core, vn, ssrc);
    const long long leaves = 1LL << w.D;
    trace_launch();
    seg_leaf_kernel<P><<<(unsigned)((leaves * 32 + 255) / 256), 256, 0, st>>>(ssrc, m, w.D, geo, box, mom);
    for (int l = w.D - 1; l >= 0; --l) {
        const long long t = 3 * (1LL << l);
        trace_launch();
        tree_up_kernel<P><<<(unsigned)((t + 127) / 128), 128, 0, st>>>(l, geo, box, mom);
    }
    v = SegTreeView{};
    v.ssrc = ssrc;
    v.geo = geo;
    v.mom = mom;
    v.m = m;
    v.D = w.D;
    // beyond sep the Vatistas core changes a segment's velocity by less than 2e-6 of
    // itself: (r_c / h)^(2n) / n at distance h from the line
    v.sep = core > 0.f ? (float)((double)core * pow(2e-6 * vn, -0.5 / vn)) : 0.f;
    v.vn = vn;
    v.core_pos = core > 0.f;
    return cudaGetLastError();
}

// Workspace of the treecode right-hand side: the particle tree, the segment tree, the
// trees' u and J, the sorted PSE copies and nu_t.
cudaError_t tree_rhs_layout(long long n, long long m, TreeRhsWs& r)
{
    r = TreeRhsWs{};
    size_t tb = 0;
    cudaError_t e = tree_workspace(n, &tb);
    if (e != cudaSuccess) return e;
    SegTreeWs sw{};
    if (m > 0 && (e = seg_tree_layout(m, sw)) != cudaSuccess) return e;
    Carve cv;
    r.tree = cv.take(tb);
    r.stree = cv.take(sw.bytes);
    r.up = cv.take((size_t)n * 3 * sizeof(float));
    r.Jp = cv.take((size_t)n * 9 * sizeof(float));
    r.sp = cv.take((size_t)n * 16);
    r.sg = cv.take((size_t)n * 16);
    r.nut = cv.take((size_t)n * sizeof(float));
    r.counter = cv.take(sizeof(int));
    r.bytes = cv.off;
    return cudaSuccess;
}

cudaError_t run_tree_rhs(const TreeRhsWs& r, char* ws, const float* pos, const float* str, long long n,
                         const float* seg_a, const float* seg_b, long long m, const vpm_params* prm, float theta,
                         int order, float* dxdt, float* dGdt, float* nu_t, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    float* up = reinterpret_cast<float*>(ws + r.up);
    float* Jp = reinterpret_cast<float*>(ws + r.Jp);
    float* nut = nu_t ? nu_t : reinterpret_cast<float*>(ws + r.nut);
    char* tws = ws + r.tree;
    cudaError_t e;
    SegTreeView sv{};
    if (m > 0) {
        SegTreeWs sw;
        if ((e = seg_tree_layout(m, sw)) != cudaSuccess) return e;
        const int vn = prm->vatistas_n;
        switch (order) {
            case 2: e = build_seg_tree<2>(sw, ws + r.stree, seg_a, seg_b, m, prm->seg_core, vn, sv, st); break;
            case 3: e = build_seg_tree<3>(sw, ws + r.stree, seg_a, seg_b, m, prm->seg_core, vn, sv, st); break;
            default: e = build_seg_tree<4>(sw, ws + r.stree, seg_a, seg_b, m, prm->seg_core, vn, sv, st); break;
        }
        if (e != cudaSuccess) return e;
    }
    e = run_tree_induce(pos, str, n, prm->sigma, theta, order, up, Jp, tws, st, m > 0 ? &sv : nullptr);
    if (e != cudaSuccess) return e;
    trace_launch();
    tree_rhs_epilogue_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        (int)n, up, Jp, nullptr, nullptr, reinterpret_cast<const float4*>(str), prm->sigma,
        prm->c_v, prm->u_inf[0], prm->u_inf[1], prm->u_inf[2], (prm->flags & VPM_STRETCH_CLASSIC) ? 1 : 0,
        (prm->flags & VPM_CHECK_FINITE) ? 1 : 0, dev_err_ptr(), dxdt, dGdt, nut);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // PSE over the tree built for these positions (still in the tree's workspace)
    TreeWs w;
    if ((e = tree_layout(n, w)) != cudaSuccess) return e;
    float4* sp = reinterpret_cast<float4*>(ws + r.sp);
    float4* sg = reinterpret_cast<float4*>(ws + r.sg);
    const int* idx = reinterpret_cast<const int*>(tws + w.idx1);
    trace_launch();
    tree_pse_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const float4*>(pos), reinterpret_cast<const float4*>(str), nut, idx, (int)n, sp, sg);
    PseArgs A{};
    A.sp = sp;
    A.sg = sg;
    A.geo = reinterpret_cast<const float4*>(tws + w.geo);
    A.idx = idx;
    A.order = reinterpret_cast<const int*>(tws + w.lord1);
    A.n = n;
    A.D = w.D;
    const double sg2 = (double)prm->sigma * prm->sigma;
    A.sep = (float)(RHO_FAR * (double)prm->sigma);
    A.cut2 = (float)((double)RHO_FAR * RHO_FAR * sg2);
    A.inv2s2 = (float)(0.5 / sg2);
    A.nu = prm->nu;
    A.pref = (float)(2.0 / sg2 * pow(2.0 * 3.14159265358979323846 * sg2, -1.5));  // (2/sigma^2) zeta's norm
    A.counter = reinterpret_cast<int*>(ws + r.counter);
    A.dGdt = dGdt;
    if ((e = cudaMemsetAsync(A.counter, 0, sizeof(int), st)) != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tree_pse_kernel, TREE_WARPS * 32, 0)) !=
        cudaSuccess)
        return e;
    const long long leaves = 1LL << w.D;
    const long long blocks =
        std::min<long long>((leaves + TREE_WARPS - 1) / TREE_WARPS, (long long)std::max(per_sm, 1) * sm_count());
    trace_launch();
    tree_pse_kernel<<<(unsigned)blocks, TREE_WARPS * 32, 0, st>>>(A);
    return cudaGetLastError();
}

}  // namespace vpm
