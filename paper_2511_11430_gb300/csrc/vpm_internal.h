// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "vpm.h"
#include "vpm_common.cuh"

namespace vpm {

constexpr int SWEEP_CW = 16;                 // warps per sweep block
constexpr int SWEEP_TPB = SWEEP_CW * 32;
constexpr int TGT_TILE = SWEEP_CW * 64;      // targets per sweep target tile: two per thread
constexpr int SWEEP_STAGES = 6;              // shared-memory source tiles in flight
constexpr int TPB = 256;          // threads per adjoint block (8 warps)
constexpr int ADJ_TILE = 512;     // particles per adjoint tile: two per thread
constexpr int SRC_TILE = 128;     // sources per particle or segment tile
constexpr int T_F4 = 4;           // float4 per packed adjoint target (control point)
constexpr float RHO_FAR = 7.0f;   // beyond 7 sigma the blob is a point vortex in FP32
constexpr int UNIT_W_P = 10;      // stream-K cost of a particle tile
constexpr int UNIT_W_S_GRAD = 26; // ... of a segment tile with gradient
constexpr int UNIT_W_S_VEL = 20;  // ... of a segment tile, velocity only

// Workspace carving: 256-byte aligned sub-buffers.
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    }
};

int sm_count();
int* dev_err_ptr();          // device error word of the current device
int sweep_blocks(bool grad, bool comp, bool stretch, bool segments = false);  // resident sweep blocks (current device)
int adjoint_blocks(bool comp);

struct SweepPlan {
    int n_tgt = 0, n_src = 0, m_seg = 0;
    int TT = 0, SP = 0, SS = 0;
    bool grad = false, comp = false;
    bool stretch = false;  // accumulate the transposed stretching J^T Gamma_i per target
    int ncomp = 0;         // logical accumulator rows (3, 14 or 17)
    bool mixed = false;  // particle and segment tiles in one launch (small problems)
    StreamK sk{};        // particle tiles, and the segment tiles when mixed (one launch)
    StreamK sks{};       // otherwise the segment tiles (a launch of their own)
    size_t off_psrc = 0, off_pbox = 0, off_ssrc = 0, off_sbox = 0, off_part = 0, off_part_s = 0, bytes = 0;
};

// Plans a particle + segment sweep onto `n_tgt` targets from a workspace carve: the
// particle tiles and the segment tiles are split stream-K in two launches (sk, sks),
// each with its own partial sums, or in one (sk) for a small problem; fills the
// sub-buffer offsets.
SweepPlan plan_sweep(int64_t n_tgt, int64_t n_src, int64_t m_seg, bool grad, bool comp, Carve& cv,
                     bool stretch = false);

// Launches packing, the sweep and the reduction/epilogue.
struct EpilogueOut {
    int mode = 0;  // 0: velocity (+gradient) outputs; 1: right-hand side
    float* u = nullptr;
    float* grad_u = nullptr;
    const float* str = nullptr;  // particle strengths (rhs)
    float sigma = 0.f, c_v = 0.f, uinf[3] = {0, 0, 0};
    int classic = 0;
    float* dxdt = nullptr;
    float* dGdt = nullptr;
    float* nu_t = nullptr;
    int check_finite = 0;
};

cudaError_t run_sweep(const SweepPlan& p, char* ws, const float* tgt, const float* src_pos, const float* src_str,
                      const float* seg_a, const float* seg_b, float sigma, float seg_core, int vatistas_n,
                      const EpilogueOut& out, cudaStream_t st);

// Particle strength exchange added into dGdt (uses the particle tile boxes of the plan).
cudaError_t run_pse(const SweepPlan& p, char* ws, const float* pos, const float* str, const float* nu_t, int n,
                    float sigma, float nu, float* dGdt, cudaStream_t st);

// Time step kernels.
cudaError_t run_cast_state(const double* x, const double* G, const float* vol, int n, float* pos, float* str,
                           cudaStream_t st);
cudaError_t run_rk3_stage(int k, double dt, double* x, double* G, double* qx, double* qG, const float* dxdt,
                          const float* dGdt, const float* vol, int n, float* pos, float* str, cudaStream_t st);

// Adjoint sweep.
size_t backward_workspace(int64_t n_src, int64_t n_tgt, bool comp);
cudaError_t run_backward(char* ws, size_t ws_bytes, const float* src_pos, const float* src_str, int n_src,
                         const float* tgt, int n_tgt, float sigma, bool comp, const float* g, float* dx, float* dG,
                         cudaStream_t st);

// AIC build and solve.
cudaError_t run_aic_build(const float* rings, const float* colloc, const float* normal, int n, float core, int vn,
                          const float* v_rel, const float* w_ind, float* A, double* b, cudaStream_t st);
cudaError_t run_selftest_wait(double limit_ms, int* completed, cudaStream_t st);
cudaError_t run_wake_segments(const double* nodes, const double* gamma, long long R, long long nb, long long S,
                              float* seg_a, float* seg_b, cudaStream_t st);
cudaError_t run_ring_segments(const float* rings, const double* gamma, long long n, float* seg_a, float* seg_b,
                              cudaStream_t st);
cudaError_t run_points_pack(const double* pts, long long n, float* tgt, cudaStream_t st);
cudaError_t run_points_advect(double* pts, const float* u, long long n, double dt, const float* u_inf, cudaStream_t st);
size_t loads_workspace(long long m, long long n);
cudaError_t run_segment_midpoints(const float* seg_a, const float* seg_b, long long m, float* tgt, cudaStream_t st);
cudaError_t run_blade_loads(const float* seg_a, const float* seg_b, long long m, const float* u_ind,
                            const double* omega, const double* hub, const double* u_inf, const float* rings,
                            const float* normal, const double* gamma, const double* gamma_prev, long long n, double dt,
                            double rho, double* out, char* ws, cudaStream_t st);
size_t wake_workspace(long long m, bool row_edges);
vpm_status run_wake_convert(const double* a, const double* b, const double* gamma, const double* gamma_nb,
                            const int* has_nb, const int* trailed, long long m, double ds_tip, int n_tip, int n_shed,
                            double* x, double* G, long long ld, long long* n_out, char* ws, cudaStream_t st,
                            const char** msg);
vpm_status run_wake_convert_row(const double* U, const double* D, const double* gamma, long long S, double ds_tip,
                                int n_tip, int n_shed, double* x, double* G, long long ld, long long* n_out, char* ws,
                                cudaStream_t st, const char** msg);
cudaError_t tree_workspace(long long n, size_t* bytes);
struct TreeRhsWs {
    size_t tree, stree, up, Jp, sp, sg, nut, counter, bytes;
};
// A built segment tree, as the treecode's traversal reads it.
struct SegTreeView {
    const float4* ssrc;  // sorted packed segments [m][S_F4]
    const float4* geo;   // per node (cx, cy, cz, r)
    const float* mom;    // per node [3][NM] scaled moments of the line strengths
    long long m;
    int D;               // depth
    float sep;           // least sphere distance of a far node
    int vn, core_pos;    // Vatistas exponent; the core is > 0
};
cudaError_t tree_rhs_layout(long long n, long long m, TreeRhsWs& r);
cudaError_t run_tree_rhs(const TreeRhsWs& r, char* ws, const float* pos, const float* str, long long n,
                         const float* seg_a, const float* seg_b, long long m, const vpm_params* prm, float theta,
                         int order, float* dxdt, float* dGdt, float* nu_t, cudaStream_t st);
cudaError_t run_tree_induce(const float* pos, const float* str, long long n, float sigma, float theta, int order,
                            float* u, float* grad_u, char* ws, cudaStream_t st, const SegTreeView* segs = nullptr);
size_t aic_workspace(int n);
vpm_status run_aic_solve(const float* A, const double* b, double* x, int n, double tol, int max_iter, int* iters,
                         double* berr, char* ws, cudaStream_t st, const char** msg);

// Launch tracing (vpm_trace_*): count launches; time the bracketed kernels.
constexpr int TRACE_KINDS = 6;
void trace_launch(int count = 1);
class TraceScope {
  public:
    TraceScope(int kind, cudaStream_t st);
    ~TraceScope();

  private:
    int kind_;
    cudaStream_t st_;
    void* a_ = nullptr;
    void* b_ = nullptr;
};

}  // namespace vpm
