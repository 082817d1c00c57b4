// Wake panel -> particle conversion (Sec. II.C, Eq. 6-8).
//
//  * An edge is one straight vortex line a -> b of the wake lattice, owned by a wake
//    panel of circulation gamma; its circulation difference is gamma - gamma_nb when
//    the panel across the edge is converted with it, else gamma (Eq. 7).
//  * A trailed edge becomes n = ceil(|b - a| / ds_tip * n_tip) particles (Eq. 8), a
//    shed edge n_shed; particle k sits at the centre of the k-th of n equal pieces and
//    carries Delta Gamma (b - a) / n (Eq. 6).
//  * Counts per edge with per-tile sums, a scan of the tile sums (and the total), the
//    offsets within each tile, and the scatter, one thread per particle.  The count is an
//    integer decided by floating point, so it is formed in double precision with
//    explicitly rounded operations (no contraction), the reading the reference takes.
#include <math.h>

#include "vpm_internal.h"

namespace vpm {

__device__ __forceinline__ long long wake_count(const double* a, const double* b, int trailed, double ds_tip,
                                                int n_tip, int n_shed)
{
    if (!trailed) return n_shed;
    if (n_tip < 0) return -(long long)n_tip;  // conventional: the same count on every trailed edge
    const double dx = __dsub_rn(b[0], a[0]), dy = __dsub_rn(b[1], a[1]), dz = __dsub_rn(b[2], a[2]);
    const double len = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    const double v = ceil(__dmul_rn(__ddiv_rn(len, ds_tip), (double)n_tip));
    // a zero-length edge keeps one particle (of zero strength); a count above the largest
    // capacity (or NaN) is clamped to VPM_MAX_ITEMS + 1, which no capacity admits, so the
    // total stays far from overflow and the call is refused
    if (!(v <= (double)VPM_MAX_ITEMS)) return (long long)VPM_MAX_ITEMS + 1;
    return v < 1.0 ? 1 : (long long)v;
}

// Counts are scanned in tiles of SCAN_TILE edges: block t of wake_count_kernel writes
// its tile's counts and their sum, one block scans the tile sums, and
// wake_offsets_kernel scans each tile and adds the tile's start.
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER;

// Inclusive scan of v over the block (SCAN_THREADS threads); returns this thread's
// inclusive prefix and puts the block total in *tot.
__device__ __forceinline__ long long block_scan(long long v, long long* wsum, long long* tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        if (lane < SCAN_THREADS / 32) wsum[lane] = w;
    }
    __syncthreads();
    const long long r = v + (warp > 0 ? wsum[warp - 1] : 0);
    *tot = wsum[SCAN_THREADS / 32 - 1];
    __syncthreads();  // wsum may be reused by the caller
    return r;
}

// Also writes every edge's particle strength Delta Gamma (b - a) / n (Eq. 6, 7): the
// same for all n particles of the edge, so it is formed once here.
__global__ void __launch_bounds__(SCAN_THREADS) wake_count_kernel(const double* __restrict__ a,
                                                                  const double* __restrict__ b,
                                                                  const double* __restrict__ gamma,
                                                                  const double* __restrict__ gamma_nb,
                                                                  const int* __restrict__ has_nb,
                                                                  const int* __restrict__ trailed, long long m,
                                                                  double ds_tip, int n_tip, int n_shed,
                                                                  long long* __restrict__ counts,
                                                                  double* __restrict__ strength,
                                                                  long long* __restrict__ tile_sum)
{
    __shared__ long long wsum[SCAN_THREADS / 32];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    long long s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        const long long i = base + k * SCAN_THREADS + threadIdx.x;
        if (i < m) {
            const long long c = wake_count(a + 3 * i, b + 3 * i, trailed[i], ds_tip, n_tip, n_shed);
            counts[i] = c;
            s += c;
            const double dG = (has_nb && has_nb[i]) ? __dsub_rn(gamma[i], gamma_nb[i]) : gamma[i];  // Eq. 7
            const double nd = (double)c;
#pragma unroll
            for (int q = 0; q < 3; ++q)
                strength[3 * i + q] = __ddiv_rn(__dmul_rn(dG, __dsub_rn(b[3 * i + q], a[3 * i + q])), nd);  // Eq. 6
        }
    }
    long long tot;
    block_scan(s, wsum, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// Exclusive scan of the tile sums (one block, looping over chunks of SCAN_THREADS), and
// the grand total.
__global__ void __launch_bounds__(SCAN_THREADS) wake_tile_scan_kernel(long long* __restrict__ tile_sum,
                                                                      long long tiles, long long* __restrict__ total)
{
    __shared__ long long wsum[SCAN_THREADS / 32];
    long long carry = 0;
    for (long long c0 = 0; c0 < tiles; c0 += SCAN_THREADS) {
        const long long i = c0 + threadIdx.x;
        const long long v = i < tiles ? tile_sum[i] : 0;
        long long tot;
        const long long incl = block_scan(v, wsum, &tot);
        if (i < tiles) tile_sum[i] = carry + incl - v;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

// offsets[i] = the tile's start + the exclusive prefix of counts within the tile.
__global__ void __launch_bounds__(SCAN_THREADS) wake_offsets_kernel(const long long* __restrict__ counts, long long m,
                                                                    const long long* __restrict__ tile_start,
                                                                    long long* __restrict__ offsets)
{
    __shared__ long long wsum[SCAN_THREADS / 32];
    const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_PER;
    long long c[SCAN_PER], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {  // a thread scans SCAN_PER consecutive edges
        c[k] = base + k < m ? counts[base + k] : 0;
        s += c[k];
    }
    long long tot;
    long long run = block_scan(s, wsum, &tot) - s + tile_start[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        if (base + k < m) offsets[base + k] = run;
        run += c[k];
    }
}

// One thread per particle p < total: its edge i is the last with offsets[i] <= p
// (binary search; edges without particles do not exist, every count is >= 1), its
// index within the edge k = p - offsets[i].  Writes are coalesced across the warp
// (planar outputs of leading dimension ld).
__global__ void wake_scatter_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                    const double* __restrict__ strength, long long m,
                                    const long long* __restrict__ counts, const long long* __restrict__ offsets,
                                    long long total, double* __restrict__ x, double* __restrict__ G, long long ld)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    long long lo = 0, hi = m - 1;  // offsets[lo] <= p < offsets[hi + 1]
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= p)
            lo = mid;
        else
            hi = mid - 1;
    }
    const long long i = lo, k = p - offsets[i];
    const double* ai = a + 3 * i;
    const double* bi = b + 3 * i;
    const double t = __ddiv_rn(__dadd_rn((double)k, 0.5), (double)counts[i]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        x[c * ld + p] = __dadd_rn(ai[c], __dmul_rn(t, __dsub_rn(bi[c], ai[c])));
        G[c * ld + p] = strength[3 * i + c];
    }
}

// The 3 S + 1 edges of one wake panel row (node lines U, D [S+1][3], circulations
// gamma [S]): trailed q < S: D[q] -> U[q] of panel q with neighbour q - 1 (q > 0);
// trailed S: U[S] -> D[S] of panel S - 1; shed back p: D[p+1] -> D[p]; shed front p:
// U[p] -> U[p+1]; shed edges without neighbour.
__global__ void wake_row_edges_kernel(const double* __restrict__ U, const double* __restrict__ D,
                                      const double* __restrict__ gamma, long long S, double* __restrict__ a,
                                      double* __restrict__ b, double* __restrict__ g, double* __restrict__ gnb,
                                      int* __restrict__ has_nb, int* __restrict__ trailed)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > 3 * S) return;
    const double *from, *to;
    double ge, gn = 0.0;
    int hn = 0, tr = 0;
    if (e <= S) {  // trailed
        const long long q = e;
        const bool end = q == S;
        from = end ? U + 3 * q : D + 3 * q;
        to = end ? D + 3 * q : U + 3 * q;
        ge = end ? gamma[S - 1] : gamma[q];
        hn = (!end && q > 0);
        if (hn) gn = gamma[q - 1];
        tr = 1;
    } else if (e <= 2 * S) {  // shed, downstream line
        const long long p = e - S - 1;
        from = D + 3 * (p + 1);
        to = D + 3 * p;
        ge = gamma[p];
    } else {  // shed, upstream line
        const long long p = e - 2 * S - 1;
        from = U + 3 * p;
        to = U + 3 * (p + 1);
        ge = gamma[p];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) a[3 * e + c] = from[c], b[3 * e + c] = to[c];
    g[e] = ge, gnb[e] = gn, has_nb[e] = hn, trailed[e] = tr;
}

// ---------------------------------------------------------------------------
// The near wake between conversions: R panel rows per blade between R + 1 node lines
// (line 0 at the trailing edge), nodes stored [line][blade][S + 1][3] in FP64.
// ---------------------------------------------------------------------------
// The four segments of every wake ring: row r, blade b, panel p is the ring
// U[p] -> U[p+1] -> D[p+1] -> D[p] -> U[p] with U = line r and D = line r + 1,
// circulation gamma[r][b][p]; segment k of the ring is out[4 ((r nb + b) S + p) + k].
__global__ void wake_segments_kernel(const double* __restrict__ nodes, const double* __restrict__ gamma, long long R,
                                     long long nb, long long S, float4* __restrict__ seg_a,
                                     float4* __restrict__ seg_b)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // panel index (r nb + b) S + p
    if (i >= R * nb * S) return;
    const long long p = i % S, rb = i / S;  // rb = r nb + b
    const long long up = rb * (S + 1) + p, dn = (rb + nb) * (S + 1) + p;
    const long long c[4] = {up, up + 1, dn + 1, dn};
    const float g = (float)gamma[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double* a = nodes + 3 * c[k];
        const double* b = nodes + 3 * c[(k + 1) & 3];
        seg_a[4 * i + k] = make_float4((float)a[0], (float)a[1], (float)a[2], g);
        seg_b[4 * i + k] = make_float4((float)b[0], (float)b[1], (float)b[2], 0.f);
    }
}

// The four segments c0 -> c1 -> c2 -> c3 -> c0 of blade rings [n][4] (float4 corners)
// carrying circulations gamma [n] (FP64, as aic_solve returns them).
__global__ void ring_segments_kernel(const float4* __restrict__ rings, const double* __restrict__ gamma, long long n,
                                     float4* __restrict__ seg_a, float4* __restrict__ seg_b)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = (float)gamma[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 a = rings[4 * i + k], b = rings[4 * i + ((k + 1) & 3)];
        seg_a[4 * i + k] = make_float4(a.x, a.y, a.z, g);
        seg_b[4 * i + k] = make_float4(b.x, b.y, b.z, 0.f);
    }
}

cudaError_t run_ring_segments(const float* rings, const double* gamma, long long n, float* seg_a, float* seg_b,
                              cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    trace_launch();
    ring_segments_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float4*>(rings), gamma, n,
                                                                      reinterpret_cast<float4*>(seg_a),
                                                                      reinterpret_cast<float4*>(seg_b));
    return cudaGetLastError();
}

// FP32 targets (x, y, z, 0) of n FP64 points [n][3].
__global__ void points_pack_kernel(const double* __restrict__ pts, long long n, float4* __restrict__ tgt)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    tgt[i] = make_float4((float)pts[3 * i], (float)pts[3 * i + 1], (float)pts[3 * i + 2], 0.f);
}

// pts[i] += dt (u[:, i] + u_inf), u planar [3][n] FP32, pts [n][3] FP64 (explicit Euler).
__global__ void points_advect_kernel(double* __restrict__ pts, const float* __restrict__ u, long long n, double dt,
                                     double ux, double uy, double uz)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pts[3 * i] += dt * ((double)u[i] + ux);
    pts[3 * i + 1] += dt * ((double)u[n + i] + uy);
    pts[3 * i + 2] += dt * ((double)u[2 * n + i] + uz);
}

cudaError_t run_wake_segments(const double* nodes, const double* gamma, long long R, long long nb, long long S,
                              float* seg_a, float* seg_b, cudaStream_t st)
{
    const long long np = R * nb * S;
    if (np == 0) return cudaSuccess;
    trace_launch();
    wake_segments_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(nodes, gamma, R, nb, S,
                                                                       reinterpret_cast<float4*>(seg_a),
                                                                       reinterpret_cast<float4*>(seg_b));
    return cudaGetLastError();
}

cudaError_t run_points_pack(const double* pts, long long n, float* tgt, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    trace_launch();
    points_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pts, n, reinterpret_cast<float4*>(tgt));
    return cudaGetLastError();
}

cudaError_t run_points_advect(double* pts, const float* u, long long n, double dt, const float* u_inf, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    trace_launch();
    points_advect_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pts, u, n, dt, u_inf ? u_inf[0] : 0.0,
                                                                      u_inf ? u_inf[1] : 0.0, u_inf ? u_inf[2] : 0.0);
    return cudaGetLastError();
}

namespace {
struct WakeWs {
    size_t counts, offsets, total, tiles, strength, ea, eb, eg, egnb, ehn, etr, bytes;
};
WakeWs wake_layout(long long m, bool row_edges)
{
    Carve cv;
    WakeWs w{};
    w.counts = cv.take((size_t)m * sizeof(long long));
    w.offsets = cv.take((size_t)m * sizeof(long long));
    w.total = cv.take(sizeof(long long));
    w.tiles = cv.take((size_t)((m + SCAN_TILE - 1) / SCAN_TILE + 1) * sizeof(long long));
    w.strength = cv.take((size_t)m * 3 * sizeof(double));
    if (row_edges) {
        w.ea = cv.take((size_t)m * 3 * sizeof(double));
        w.eb = cv.take((size_t)m * 3 * sizeof(double));
        w.eg = cv.take((size_t)m * sizeof(double));
        w.egnb = cv.take((size_t)m * sizeof(double));
        w.ehn = cv.take((size_t)m * sizeof(int));
        w.etr = cv.take((size_t)m * sizeof(int));
    }
    w.bytes = cv.off;
    return w;
}
}  // namespace

size_t wake_workspace(long long m, bool row_edges) { return wake_layout(m, row_edges).bytes; }

vpm_status run_wake_convert(const double* a, const double* b, const double* gamma, const double* gamma_nb,
                            const int* has_nb, const int* trailed, long long m, double ds_tip, int n_tip, int n_shed,
                            double* x, double* G, long long ld, long long* n_out, char* ws, cudaStream_t st,
                            const char** msg)
{
    const WakeWs L = wake_layout(m, false);
    long long* counts = reinterpret_cast<long long*>(ws + L.counts);
    long long* offsets = reinterpret_cast<long long*>(ws + L.offsets);
    long long* total = reinterpret_cast<long long*>(ws + L.total);
    long long* tiles = reinterpret_cast<long long*>(ws + L.tiles);
    const long long ntiles = (m + SCAN_TILE - 1) / SCAN_TILE;
    trace_launch();
    double* strength = reinterpret_cast<double*>(ws + L.strength);
    wake_count_kernel<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(a, b, gamma, gamma_nb, has_nb, trailed, m, ds_tip,
                                                                 n_tip, n_shed, counts, strength, tiles);
    trace_launch();
    wake_tile_scan_kernel<<<1, SCAN_THREADS, 0, st>>>(tiles, ntiles, total);
    trace_launch();
    wake_offsets_kernel<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(counts, m, tiles, offsets);
    long long h = 0;
    if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&h, total, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        *msg = cudaGetErrorString(cudaGetLastError());
        return VPM_ERR_CUDA;
    }
    *n_out = h;
    if (h > ld || h > VPM_MAX_ITEMS) {
        *msg = "wake_convert: more particles than the output capacity ld_out";
        return VPM_ERR_LIMIT;
    }
    if (h == 0) return VPM_OK;
    const int tpb = 256;
    trace_launch();
    wake_scatter_kernel<<<(unsigned)((h + tpb - 1) / tpb), tpb, 0, st>>>(a, b, strength, m, counts, offsets, h, x,
                                                                      G, ld);
    if (cudaGetLastError() != cudaSuccess) {
        *msg = cudaGetErrorString(cudaGetLastError());
        return VPM_ERR_CUDA;
    }
    return VPM_OK;
}

vpm_status run_wake_convert_row(const double* U, const double* D, const double* gamma, long long S, double ds_tip,
                                int n_tip, int n_shed, double* x, double* G, long long ld, long long* n_out, char* ws,
                                cudaStream_t st, const char** msg)
{
    const long long m = 3 * S + 1;
    const WakeWs L = wake_layout(m, true);
    double* a = reinterpret_cast<double*>(ws + L.ea);
    double* b = reinterpret_cast<double*>(ws + L.eb);
    double* g = reinterpret_cast<double*>(ws + L.eg);
    double* gnb = reinterpret_cast<double*>(ws + L.egnb);
    int* hn = reinterpret_cast<int*>(ws + L.ehn);
    int* tr = reinterpret_cast<int*>(ws + L.etr);
    trace_launch();
    wake_row_edges_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(U, D, gamma, S, a, b, g, gnb, hn, tr);
    if (cudaGetLastError() != cudaSuccess) {
        *msg = cudaGetErrorString(cudaGetLastError());
        return VPM_ERR_CUDA;
    }
    // the edge arrays sit after the conversion's own scratch in the same layout
    return run_wake_convert(a, b, g, gnb, hn, tr, m, ds_tip, n_tip, n_shed, x, G, ld, n_out, ws, st, msg);
}

}  // namespace vpm
