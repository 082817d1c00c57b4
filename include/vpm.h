/*
 * vpm.h -- C ABI of the GB300 (sm_103a) vortex-particle hot path of the
 * NL-UVLM-VPM rotor-wake method (Fu & Laurendeau, arXiv 2511.11430).
 *
 * The library evaluates the Gaussian-regularised Biot-Savart velocity u and
 * velocity gradient grad u on vortex particles (Sec. II.B, Eq. 2-4) from all
 * other particles and from Vatistas-cored straight vortex segments (Sec. II.A),
 * the vortex-particle right-hand side of Eq. 4-5 (stretching, PSE diffusion with
 * the Vreman eddy viscosity), one low-storage third-order Runge-Kutta step, the
 * blade influence-coefficient (AIC) system with FP32 LU and FP64 iterative
 * refinement, and the adjoint of the particle-to-point velocity.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named *_d are DEVICE pointers on the current CUDA device; the
 *    caller owns every buffer.  The library allocates nothing and frees nothing;
 *    scratch memory is the caller's `ws` of at least vpm_workspace_size() bytes.
 *  - float4-packed arrays are `const float*` with 4 floats per item, 16-byte
 *    aligned:  particles  pos[n][4] = (x, y, z, volume)   str[n][4] = (Gx, Gy, Gz, -)
 *              targets    tgt[n][4] = (x, y, z, -)
 *              segments   seg_a[m][4] = (ax, ay, az, circulation)   seg_b[m][4] = (bx, by, bz, -)
 *    The 4th lane marked "-" is ignored.
 *  - Outputs are planar: u[3][n] (u[a*n + i]), grad_u[9][n] with
 *    grad_u[(3*a+b)*n + i] = d u_a / d x_b at target i.
 *  - SI units as in the paper: lengths in m, particle strength Gamma in m^3/s,
 *    segment circulation in m^2/s.
 *  - A pair at zero distance contributes nothing, so a particle never induces
 *    velocity on itself when the targets are the particles.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Entry points are asynchronous on that stream unless stated otherwise.
 *  - Return codes report argument errors (nothing is launched) and launch
 *    errors.  Faults found by kernels (a bounded wait that timed out, a
 *    non-finite output when VPM_CHECK_FINITE is set) are latched in a device
 *    word read by vpm_device_error().
 *  - Calls on different streams must not share a workspace.
 *  - Per-device set-up done once (the treecode's interpolation table) does not
 *    survive cudaDeviceReset: after resetting a device, reload the library before
 *    using it on that device again.
 */
#ifndef VPM_H
#define VPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vpm_status {
    VPM_OK = 0,
    VPM_ERR_INVALID_ARG = -1,   /* bad size, NULL or misaligned pointer, sigma <= 0 ... */
    VPM_ERR_CUDA = -2,          /* a CUDA runtime call or kernel launch failed */
    VPM_ERR_NONFINITE = -3,     /* a kernel saw a non-finite value (device word) */
    VPM_ERR_NOT_CONVERGED = -4, /* aic_solve: backward error above tol after max_iter */
    VPM_ERR_WORKSPACE = -5,     /* ws NULL or smaller than vpm_workspace_size() */
    VPM_ERR_LIMIT = -6          /* a size above the library's limits */
} vpm_status;

/* flags (bitwise or) */
#define VPM_COMPENSATED 0x1     /* compensated FP32 accumulation (two-sum per source tile) */
#define VPM_STRETCH_CLASSIC 0x2 /* stretching (Gamma . grad) u = J Gamma (Eq. 1) instead of
                                   the transposed (Gamma . grad^T) u = J^T Gamma of Eq. 5 */
#define VPM_CHECK_FINITE 0x4    /* scan outputs for NaN/Inf and latch VPM_ERR_NONFINITE */

/* operation codes for vpm_workspace_size */
#define VPM_OP_INDUCE 1
#define VPM_OP_SEGMENTS 2
#define VPM_OP_RHS 3
#define VPM_OP_STEP 4
#define VPM_OP_AIC_SOLVE 5
#define VPM_OP_BACKWARD 6
#define VPM_OP_WAKE_CONVERT 7
#define VPM_OP_WAKE_ROW 8
#define VPM_OP_LOADS 9
#define VPM_OP_TREE 10
#define VPM_OP_RHS_TREE 11
#define VPM_OP_STEP_TREE 12
#define VPM_OP_STAGE 13

/* Largest particle / target / segment count accepted (int32 indexing). */
#define VPM_MAX_ITEMS (1 << 30)
/* Largest AIC order accepted by aic_solve. */
#define VPM_MAX_AIC 8192

/* Parameters of the vortex-particle right-hand side (Sec. II.B). */
typedef struct vpm_params {
    float sigma;      /* particle core size sigma of Eq. 3 [m], > 0 */
    float nu;         /* kinematic viscosity [m^2/s], >= 0 */
    float c_v;        /* Vreman coefficient (the paper uses 0.07), >= 0 */
    float seg_core;   /* Vatistas core radius of the segments [m], >= 0 */
    float u_inf[3];   /* free-stream velocity added to dx/dt [m/s] */
    int vatistas_n;   /* Vatistas exponent n, 1 or 2 */
    int flags;        /* VPM_COMPENSATED | VPM_STRETCH_CLASSIC | VPM_CHECK_FINITE */
} vpm_params;

/* Message of the last error returned on the calling host thread ("" if none). */
const char* vpm_last_error(void);

/* ABI version (major * 10000 + minor * 100 + patch).  1.1: vpm_rk3_stage,
 * VPM_OP_STAGE and the segment trace kind VPM_TRACE_SEGMENTS. */
int vpm_version(void);

/* Reads and clears the device error word of the current device (synchronises the
 * device).  *code receives 0, VPM_ERR_NONFINITE, or VPM_ERR_LIMIT (a bounded wait
 * inside a kernel timed out).  Returns VPM_ERR_CUDA if the read itself fails. */
vpm_status vpm_device_error(int* code);

/* Bytes of scratch an operation needs on the current device.
 *   VPM_OP_INDUCE:    n_src particles -> n_tgt targets            (m_seg ignored)
 *   VPM_OP_SEGMENTS:  m_seg segments -> n_tgt targets             (n_src ignored)
 *   VPM_OP_RHS, VPM_OP_STEP: n_src particles, m_seg segments       (n_tgt ignored)
 *   VPM_OP_AIC_SOLVE: order n_tgt                                  (others ignored)
 *   VPM_OP_BACKWARD:  n_src particles, n_tgt targets
 *   VPM_OP_WAKE_CONVERT: n_src edges;  VPM_OP_WAKE_ROW: n_src panels of the row
 *   VPM_OP_LOADS:     m_seg bound segments, n_tgt panels
 *   VPM_OP_TREE:      n_src particles (vpm_tree_induce)
 *   VPM_OP_RHS_TREE, VPM_OP_STEP_TREE: n_src particles, m_seg segments
 *   VPM_OP_STAGE:     n_src particles, m_seg segments (vpm_rk3_stage)
 * `flags` as passed to the operation.  Host-only; does not launch. */
vpm_status vpm_workspace_size(int op, int64_t n_src, int64_t n_tgt, int64_t m_seg, int flags, size_t* bytes);

/* ---- Eq. 2-4: Gaussian-particle velocity and velocity gradient -----------
 * u(x) = sum_j K(r) Gamma_j x r,  r = x - x_j,  K = g(|r|/sigma) / (4 pi |r|^3),
 * g(rho) = erf(rho/sqrt2) - sqrt(2/pi) rho exp(-rho^2/2) the vorticity fraction of
 * a Gaussian blob (Eq. 3) inside radius rho*sigma; grad_u is its exact gradient.
 *   src_pos_d, src_str_d  [n_src][4]   sources (volume lane unused here)
 *   tgt_d                 [n_tgt][4]   evaluation points (may alias src_pos_d)
 *   u_d                   [3][n_tgt]   output velocity
 *   grad_u_d              [9][n_tgt]   output gradient, or NULL for velocity only
 *   flags: VPM_COMPENSATED, VPM_CHECK_FINITE.
 * n_src == 0 writes zeros; n_tgt == 0 does nothing. */
vpm_status vpm_induce(const float* src_pos_d, const float* src_str_d, int64_t n_src, const float* tgt_d,
                      int64_t n_tgt, float sigma, int flags, float* u_d, float* grad_u_d, void* ws_d,
                      size_t ws_bytes, void* stream);

/* ---- Sec. II.B: the fast summation, as a treecode --------------------------
 * u and grad u at every particle from all the others, as vpm_induce with the
 * particles as targets, in O(n log n) work.  Sec. II.B evaluates these sums with a
 * Cartesian fast multipole method; this is its treecode form: far clusters enter by
 * the Cartesian Taylor expansion of the point-vortex potential sum_j Gamma_j / |x - x_j|
 * to order `order` (moments up to |k| = order), near ones by the direct sum.
 * Clusters are runs of the particles sorted along a Morton curve, halved down to
 * leaves of at most 64; a cluster is far from a target leaf when the sum of their
 * radii is below theta times the distance of their centres and every pair is at
 * least 7 sigma apart (where the Gaussian blob equals the point vortex in FP32).
 * theta = 0 opens every cluster: the direct sum (plain FP32 accumulation).  The
 * truncation error falls as theta^(order + 1).
 * Near pairs take the blob kernel from a 16 KB table (cubic Hermite interpolation in
 * rho^2, error far below FP32 rounding); the first call on each device copies that
 * table to the device synchronously, so make it before any stream capture.
 *   pos_d, str_d [n][4] particles; u_d [3][n]; grad_u_d [9][n] or NULL;
 *   0 <= theta <= 1; order in {2, 3, 4}.  Workspace: VPM_OP_TREE (n_src = n). */
vpm_status vpm_tree_induce(const float* pos_d, const float* str_d, int64_t n, float sigma, float theta, int order,
                           float* u_d, float* grad_u_d, void* ws_d, size_t ws_bytes, void* stream);

/* The right-hand side of Eq. 4-5 (as vpm_rhs) and one RK3 step (as vpm_step) with the
 * particle-particle u and grad u from the treecode of vpm_tree_induce (theta, order as
 * there) instead of the direct sweep.  The segments form a second tree (by midpoint):
 * a node far from a target leaf enters its local expansion through the moments of the
 * segments' line strengths (exact through order 5 by 3-point Gauss-Legendre), where
 * "far" also requires the node to be at least core (2e-6 n)^(-1/(2n)) away (there the
 * Vatistas core changes the velocity by < 2e-6); nearer segments use the exact kernel
 * of vpm_segments_induce.  All sums accumulate in plain FP32 (VPM_COMPENSATED has no
 * effect here).  Vreman's eddy viscosity
 * and the stretching are formed in FP64 from the summed u and grad u (the transposed
 * stretching from J^T Gamma, not pair by pair), and the PSE term is summed over the
 * pairs within 7 sigma found by a walk of the same tree.  theta = 0 gives the direct
 * sums.  For particle counts where the direct sweep's O(n^2) cost dominates (1e6 and
 * more).  Workspace: VPM_OP_RHS_TREE / VPM_OP_STEP_TREE (n_src = n, m_seg = m). */
vpm_status vpm_rhs_tree(const float* pos_d, const float* str_d, int64_t n, const float* seg_a_d, const float* seg_b_d,
                        int64_t m, const vpm_params* prm, float theta, int order, float* dxdt_d, float* dGdt_d,
                        float* nu_t_d, void* ws_d, size_t ws_bytes, void* stream);
vpm_status vpm_step_tree(double* x_d, double* G_d, const float* vol_d, int64_t n, const float* seg_a_d,
                         const float* seg_b_d, int64_t m, const vpm_params* prm, float theta, int order, double dt,
                         void* ws_d, size_t ws_bytes, void* stream);

/* ---- Sec. II.A: straight vortex segments with a Vatistas core ------------
 * The finite-segment Biot-Savart law with |r1 x r2|^2 replaced by
 * (|r1 x r2|^(2n) + (core |b - a|)^(2n))^(1/n), n = vatistas_n in {1, 2}, and its
 * exact gradient.  Points within 1e-10 |b-a| (or 1e-15 m) of an end point, and
 * points on the line when core == 0, receive nothing from that segment.
 *   seg_a_d, seg_b_d [m][4] (circulation in seg_a's 4th lane); tgt_d [n_tgt][4];
 *   u_d [3][n_tgt]; grad_u_d [9][n_tgt] or NULL.  flags: VPM_COMPENSATED. */
vpm_status vpm_segments_induce(const float* seg_a_d, const float* seg_b_d, int64_t m, const float* tgt_d,
                               int64_t n_tgt, float core, int vatistas_n, int flags, float* u_d, float* grad_u_d,
                               void* ws_d, size_t ws_bytes, void* stream);

/* ---- Eq. 4-5: vortex-particle right-hand side -----------------------------
 * For every particle i (targets = sources = the n particles):
 *   u_i, J_i   from all other particles (Eq. 2-4) plus the m segments
 *   nu_t,i     Vreman (2004): c_V sqrt(B_beta / alpha:alpha), alpha = J^T,
 *              beta = sigma^2 J J^T (filter width = sigma)
 *   dx/dt      = u_i + u_inf
 *   dGamma/dt  = J_i^T Gamma_i (or J_i Gamma_i with VPM_STRETCH_CLASSIC)
 *              + (2/sigma^2) sum_j nu_ij (v_i Gamma_j - v_j Gamma_i) zeta_sigma(r_ij)
 *                with nu_ij = nu + (nu_t,i + nu_t,j)/2 (particle strength exchange,
 *                pairs beyond 7 sigma skipped: zeta there is below 3e-11 of its peak)
 *   pos_d, str_d [n][4] (volume v_i in pos's 4th lane); seg_a_d/seg_b_d may be NULL if m == 0.
 *   dxdt_d, dGdt_d [3][n]; nu_t_d [n] or NULL. */
vpm_status vpm_rhs(const float* pos_d, const float* str_d, int64_t n, const float* seg_a_d, const float* seg_b_d,
                   int64_t m, const vpm_params* prm, float* dxdt_d, float* dGdt_d, float* nu_t_d, void* ws_d,
                   size_t ws_bytes, void* stream);

/* ---- FP64 master state -> FP32 packed particles (the RK state of Sec. II.B) ---
 *   x_d, G_d [3][n] double; vol_d [n] float  ->  pos_d [n][4] = (x, y, z, vol),
 *   str_d [n][4] = (Gx, Gy, Gz, 0), each value rounded to nearest float. */
vpm_status vpm_pack_state(const double* x_d, const double* G_d, const float* vol_d, int64_t n, float* pos_d,
                          float* str_d, void* stream);

/* ---- one time step: low-storage RK3 of Williamson (1980) -------------------
 * for k = 1..3:  q <- A_k q + dt f(y);  y <- y + B_k q,
 * A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15), y = (x, Gamma) in FP64, the
 * right-hand side f evaluated by vpm_rhs on the state rounded to FP32.  Segments
 * stay frozen during the step.
 *   x_d, G_d [3][n] double, updated in place; vol_d [n] float particle volumes. */
vpm_status vpm_step(double* x_d, double* G_d, const float* vol_d, int64_t n, const float* seg_a_d,
                    const float* seg_b_d, int64_t m, const vpm_params* prm, double dt, void* ws_d, size_t ws_bytes,
                    void* stream);

/* One stage k in {0, 1, 2} of vpm_step's low-storage RK3, with the register q kept
 * by the caller between stages:
 *   q <- A_k q + dt f(y);  y <- y + B_k q      (A_0 = 0: stage 0 does not read q),
 * f evaluated by vpm_rhs on the state rounded to FP32.  Calls with k = 0, 1, 2 in turn
 * on the same q run the kernels of one vpm_step in the same order and give its
 * result bit for bit; a caller can put other work between the stages (the blade
 * circulation solve of Sec. II.A, for instance).
 *   x_d, G_d [3][n] double, updated in place; q_d [6][n] double (rows 0-2 for x,
 *   3-5 for Gamma), read for k > 0 and written; vol_d [n] float; segments as
 *   vpm_rhs.  Workspace: VPM_OP_STAGE (n_src = n, m_seg = m). */
vpm_status vpm_rk3_stage(int k, double* x_d, double* G_d, double* q_d, const float* vol_d, int64_t n,
                         const float* seg_a_d, const float* seg_b_d, int64_t m, const vpm_params* prm, double dt,
                         void* ws_d, size_t ws_bytes, void* stream);

/* ---- Sec. II.A: blade influence-coefficient system -------------------------
 * A[k][l] = u(ring l, unit circulation)(y_k) . n_k with ring l the four segments
 * c0->c1->c2->c3->c0 of its corners (Vatistas core `core`, exponent vatistas_n),
 * and, when b_d is not NULL, b[k] = -(v_rel[k] + w_ind[k]) . n_k (Neumann condition).
 *   rings_d [n][4][4] corners (xyz, -); colloc_d, normal_d, v_rel_d [n][4];
 *   w_ind_d [3][n] or NULL; A_d [n][n] float row-major; b_d [n] double or NULL. */
vpm_status aic_build(const float* rings_d, const float* colloc_d, const float* normal_d, int n, float core,
                     int vatistas_n, const float* v_rel_d, const float* w_ind_d, float* A_d, double* b_d,
                     void* stream);

/* Solves A x = b with A factored once in FP32 and iterative refinement whose residual
 * r = b - A x is formed in FP64 from the FP32 matrix.  The factorisation runs without
 * row exchanges first (for a matrix strictly diagonally dominant by rows, such as the
 * blade systems, elimination keeps every pivot nonzero and the growth at most 2); the
 * dominance test (FP64 row sums) is read with the first residual, and any other matrix
 * is then factored again with partial pivoting.  Stops when the normwise backward error
 * ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) <= tol, or after max_iter
 * corrections (then VPM_ERR_NOT_CONVERGED with the best x written); a zero pivot of the
 * pivoted factorisation also returns VPM_ERR_NOT_CONVERGED.  Synchronises `stream` once
 * per refinement step (once more for a matrix that is not row-dominant).
 *   A_d [n][n] float row-major (not modified); b_d, x_d [n] double;
 *   iters_out, berr_out host pointers or NULL. */
vpm_status aic_solve(const float* A_d, const double* b_d, double* x_d, int n, double tol, int max_iter,
                     int* iters_out, double* berr_out, void* ws_d, size_t ws_bytes, void* stream);

/* ---- adjoint of the particle -> point velocity ----------------------------
 * Given g_k = dL/du_k at the targets, returns for every source particle j
 *   dL/dGamma_j = sum_k K(r) (r x g_k)
 *   dL/dx_j     = sum_k [K(r) (Gamma_j x g_k) - H(r) ((Gamma_j x r) . g_k) r]
 * with r = y_k - x_j, H = K'(r)/r.  Pair terms are recomputed, nothing stored.
 *   grad_out_d [3][n_tgt]; dL_dx_d, dL_dG_d [3][n_src].  flags: VPM_COMPENSATED. */
vpm_status vpm_induce_backward(const float* src_pos_d, const float* src_str_d, int64_t n_src, const float* tgt_d,
                               int64_t n_tgt, float sigma, int flags, const float* grad_out_d, float* dL_dx_d,
                               float* dL_dG_d, void* ws_d, size_t ws_bytes, void* stream);

/* ---- the near wake between conversions (Sec. II.C) -------------------------
 * A near wake of R panel rows per blade (nb blades, S panels across the span) lies
 * between R + 1 node lines, line 0 at the blades' trailing edges; nodes_d holds them as
 * [R + 1][nb][S + 1][3] double.  Row r, blade b, panel p is the ring
 * U[p] -> U[p+1] -> D[p+1] -> D[p] -> U[p] (U = line r, D = line r + 1) of circulation
 * gamma_d[(r nb + b) S + p] -- the convention of vpm_wake_convert_row, so the oldest
 * row of blade b converts with U = nodes_d + 3 (S+1) ((R-1) nb + b) and
 * D = nodes_d + 3 (S+1) (R nb + b).
 * vpm_wake_segments writes the 4 R nb S segments of the rings for the velocity
 * kernels (ring segment k of panel i at 4 i + k; seg_a.w = circulation, FP32). */
vpm_status vpm_wake_segments(const double* nodes_d, const double* gamma_d, int64_t R, int64_t nb, int64_t S,
                             float* seg_a_d, float* seg_b_d, void* stream);

/* The segments c0 -> c1 -> c2 -> c3 -> c0 of n blade rings (rings_d [n][4][4] float,
 * corners as for aic_build) carrying the circulations gamma_d [n] double that aic_solve
 * returns: segment k of ring i at 4 i + k, seg_a.w = circulation (FP32). */
vpm_status vpm_ring_segments(const float* rings_d, const double* gamma_d, int64_t n, float* seg_a_d, float* seg_b_d,
                             void* stream);

/* Points [n][3] double (wake nodes) as FP32 targets [n][4] = (x, y, z, 0). */
vpm_status vpm_points_pack(const double* pts_d, int64_t n, float* tgt_d, void* stream);

/* pts[i] += dt (u[:, i] + u_inf): explicit Euler convection of points [n][3] double by
 * the velocity u_d [3][n] float (planar, as vpm_induce writes it); u_inf a host
 * float[3] or NULL. */
vpm_status vpm_points_advect(double* pts_d, const float* u_d, int64_t n, double dt, const float* u_inf,
                             void* stream);

/* ---- blade loads (Sec. II.A) ----------------------------------------------
 * Steady part by the Kutta-Joukowski theorem on every bound segment s (panel side),
 *   F_s = rho Gamma_s (V_s x (b_s - a_s)),  V_s = u_inf - omega x (mid_s - hub) + u_ind(mid_s),
 * unsteady part at every panel p (unsteady Bernoulli),
 *   F_p = rho (gamma_p - gamma_prev_p) / dt  A_p n_p,  A_p = |(c2 - c0) x (c3 - c1)| / 2,
 * summed (FP64, fixed order) into out_d[0..2] = force and out_d[3..5] = moment about
 * hub.  The caller lists the bound segments: every blade ring's sides with the ring's
 * circulation (vpm_ring_segments), so that shared sides carry their net circulation,
 * with the trailing-edge sides given zero circulation (their net circulation with the
 * wake row shed at the same step vanishes: Kutta condition).
 *   seg_a_d, seg_b_d [m][4] float (a.w = circulation); u_ind_d [3][m] float, the
 *   induced velocity at the midpoints (vpm_segment_midpoints gives the targets);
 *   omega, hub, u_inf host double[3]; rings_d [n][4][4] float, normal_d [n][4]
 *   float, gamma_d, gamma_prev_d [n] double (gamma_prev_d NULL: no unsteady part);
 *   out_d 6 doubles on the device.  Workspace: VPM_OP_LOADS. */
vpm_status vpm_blade_loads(const float* seg_a_d, const float* seg_b_d, int64_t m, const float* u_ind_d,
                           const double* omega, const double* hub, const double* u_inf, const float* rings_d,
                           const float* normal_d, const double* gamma_d, const double* gamma_prev_d, int64_t n,
                           double dt, double rho, double* out_d, void* ws_d, size_t ws_bytes, void* stream);

/* FP32 targets [m][4] = (midpoint, 0) of m segments. */
vpm_status vpm_segment_midpoints(const float* seg_a_d, const float* seg_b_d, int64_t m, float* tgt_d, void* stream);

/* ---- self-test of the bounded device waits (no counterpart in the paper) -----
 * Every wait inside the library's kernels (on an mbarrier phase) gives up after a
 * time limit, latches VPM_ERR_LIMIT in the device error word and lets the kernel
 * return.  This launches one wait on a phase that nothing completes, with a limit of
 * limit_ms (0 < limit_ms <= 2000), and synchronises `stream`: *completed (host)
 * receives 0 when the wait gave up as it must, 1 if the phase completed.  The timeout
 * is then reported (and cleared) by vpm_device_error.  Allocates nothing. */
vpm_status vpm_selftest_wait(double limit_ms, int* completed, void* stream);

/* ---- wake panel -> particle conversion (Sec. II.C, Eq. 6-8) ----------------
 * Edge i is a straight vortex line a_i -> b_i of the wake lattice, owned by a wake
 * panel of circulation gamma_i (its ring's circulation runs along a_i -> b_i).
 * Delta Gamma_i = gamma_i - gamma_nb_i if has_nb_i (the panel across the edge is
 * converted too), else gamma_i (Eq. 7).  A trailed (streamwise) edge becomes
 *   n_i = ceil(|b_i - a_i| / ds_tip * n_tip)                         (Eq. 8)
 * particles, ds_tip being the length of the tip's trailed edge, which gets n_tip; a
 * shed (spanwise) edge becomes n_shed particles.  n_tip < 0 selects the conventional
 * strategy the paper compares against: -n_tip particles on every trailed edge.  The
 * particles of an edge sit at the centres of its n_i equal pieces,
 *   x_ik = a_i + (k + 1/2)/n_i (b_i - a_i),  Gamma_ik = Delta Gamma_i (b_i - a_i) / n_i   (Eq. 6),
 * and are written edge after edge.  n_i is decided in FP64 with correctly rounded
 * operations, as (|b - a| / ds_tip) * n_tip with |b - a| = sqrt((dx dx + dy dy) + dz dz).
 *   edge_a_d, edge_b_d [m][3] double; gamma_d [m] double; gamma_nb_d [m] double and
 *   has_nb_d [m] int, both NULL when no edge has a converted neighbour; trailed_d [m]
 *   int (1 trailed, 0 shed); ds_tip > 0; n_tip != 0; n_shed >= 1.
 *   x_d, G_d [3][ld_out] double, planar (row c holds component c), the particle
 *   positions and strengths; *n_out (host) receives the particle count.
 * More particles than ld_out gives VPM_ERR_LIMIT with nothing written (and *n_out the
 * count that would be needed).  Synchronises `stream` once (to read the count). */
vpm_status vpm_wake_convert(const double* edge_a_d, const double* edge_b_d, const double* gamma_d,
                            const double* gamma_nb_d, const int* has_nb_d, const int* trailed_d, int64_t m,
                            double ds_tip, int n_tip, int n_shed, double* x_d, double* G_d, int64_t ld_out,
                            int64_t* n_out, void* ws_d, size_t ws_bytes, void* stream);

/* The same conversion for one wake panel row (the oldest row of the near wake).  The
 * row has S >= 1 panels between an upstream node line U[0..S] (towards the blade)
 * and a downstream line D[0..S]; panel p is the ring U[p] -> U[p+1] -> D[p+1] ->
 * D[p] -> U[p] of circulation gamma[p].  Its 3 S + 1 edges, in this order:
 *   trailed q = 0..S-1: D[q] -> U[q] of panel q, neighbour panel q-1 when q > 0;
 *   trailed S:          U[S] -> D[S] of panel S-1;
 *   shed p = 0..S-1:    D[p+1] -> D[p] of panel p (the older row is particles already);
 *   shed p = 0..S-1:    U[p] -> U[p+1] of panel p (the younger row stays a panel row
 *                       and keeps its own ring, so this line carries gamma[p] alone).
 *   U_d, D_d [S+1][3] double; gamma_d [S] double; other arguments as vpm_wake_convert. */
vpm_status vpm_wake_convert_row(const double* U_d, const double* D_d, const double* gamma_d, int64_t S, double ds_tip,
                                int n_tip, int n_shed, double* x_d, double* G_d, int64_t ld_out, int64_t* n_out,
                                void* ws_d, size_t ws_bytes, void* stream);

/* ---- velocity sweep without a caller workspace ------------------------------
 * The paper has no counterpart: this is a library convenience.  vpm_induce for
 * callers that cannot allocate device memory to pass as a workspace -- a solver in
 * C or Fortran linked without any CUDA memory manager, or a time-critical loop
 * that must not allocate.  Arguments and results are those of vpm_induce; the
 * scratch is a fixed VPM_NOALLOC_SCRATCH_BYTES array in the library's own device
 * memory, held by every GPU that loads the library until the process exits.
 *  - Every call looks the array's device address up on the current device; the
 *    first call on a device also loads the library's device code there, so make
 *    that first call before any stream capture.
 *  - Problems whose scratch would exceed the array return VPM_ERR_LIMIT (message
 *    in vpm_last_error) without launching anything.  The scratch of n_src sources
 *    onto n_tgt targets is about 80 bytes per source plus 112 KiB per target tile
 *    of 1,024 and per resident sweep block (one block per SM) with the gradient in
 *    compensated mode (56 KiB plain; 24 and 12 KiB velocity only): on a 152-SM
 *    GB300 up to about 250,000 particles onto themselves with the gradient
 *    (compensated) fit.
 *  - Every call uses the same array and nothing in it needs to start at zero;
 *    calls whose GPU work overlaps (other streams, other host threads) race on it
 *    and must be ordered by the caller.
 *  - It allocates nothing and frees nothing. */
#define VPM_NOALLOC_SCRATCH_BYTES (64 << 20)
vpm_status vpm_induce_noalloc(const float* src_pos_d, const float* src_str_d, int64_t n_src, const float* tgt_d,
                              int64_t n_tgt, float sigma, int flags, float* u_d, float* grad_u_d, void* stream);

/* ---- launch tracing (not part of the method; for measurement) ------------
 * Every kernel the library launches increments a host-side counter.  With
 * vpm_trace_enable(1) the pair-sweep kernels are also bracketed by CUDA events
 * recorded on their launch stream; vpm_trace_read synchronises on those events and
 * returns how many launches of `kind` were timed and their summed device time.
 * kind VPM_TRACE_ALL returns the total launch count of every kernel since the
 * last reset (and the summed time of all timed kinds).  Thread-safe. */
#define VPM_TRACE_ALL 0
#define VPM_TRACE_SWEEP 1     /* forward particle pair sweep with gradient (small problems: with the segments) */
#define VPM_TRACE_ADJOINT 2   /* adjoint pair sweep */
#define VPM_TRACE_PSE 3       /* particle strength exchange */
#define VPM_TRACE_SWEEP_VEL 4 /* forward particle pair sweep, velocity only (the same) */
#define VPM_TRACE_SEGMENTS 5  /* forward segment pair sweep (its own launch; with or without gradient) */
vpm_status vpm_trace_enable(int timing);
vpm_status vpm_trace_reset(void);
vpm_status vpm_trace_read(int kind, int64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif
#endif /* VPM_H */
