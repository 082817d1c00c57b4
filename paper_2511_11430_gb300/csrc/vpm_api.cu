// C ABI entry points: argument validation, workspace carving and launch order.
// Every arithmetic step runs in the kernels of the other translation units.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>
#include <string>

#include "vpm.h"
#include "vpm_internal.h"

using namespace vpm;

namespace {

thread_local std::string g_last_error;

vpm_status fail(vpm_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

vpm_status ok()
{
    g_last_error.clear();
    return VPM_OK;
}

vpm_status cuda_fail(cudaError_t e, const char* where)
{
    return fail(VPM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }
bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

#define REQUIRE(cond, ...)                                          \
    do {                                                            \
        if (!(cond)) return fail(VPM_ERR_INVALID_ARG, __VA_ARGS__); \
    } while (0)

vpm_status check_count(int64_t n, const char* what)
{
    if (n < 0) return fail(VPM_ERR_INVALID_ARG, "%s: negative count %lld", what, (long long)n);
    if (n > VPM_MAX_ITEMS) return fail(VPM_ERR_LIMIT, "%s: count %lld above %d", what, (long long)n, VPM_MAX_ITEMS);
    return VPM_OK;
}

size_t rhs_extra(int64_t n) { return ((size_t)n * sizeof(float) + 255) & ~size_t(255); }

struct StepWs {
    SweepPlan p;
    size_t nut, pos, str, dxdt, dGdt, qx, qG, bytes;
};

StepWs step_layout(int64_t n, int64_t m, bool comp, bool classic)
{
    StepWs s;
    Carve cv;
    s.p = plan_sweep(n, n, m, true, comp, cv, !classic);
    s.nut = cv.take((size_t)n * sizeof(float));
    s.pos = cv.take((size_t)n * 16);
    s.str = cv.take((size_t)n * 16);
    s.dxdt = cv.take((size_t)n * 3 * sizeof(float));
    s.dGdt = cv.take((size_t)n * 3 * sizeof(float));
    s.qx = cv.take((size_t)n * 3 * sizeof(double));
    s.qG = cv.take((size_t)n * 3 * sizeof(double));
    s.bytes = cv.off;
    return s;
}

// Scratch of one vpm_rk3_stage call: the sweep, nu_t, the packed state and the
// right-hand side (the RK register q belongs to the caller).
struct StageWs {
    SweepPlan p;
    size_t nut, pos, str, dxdt, dGdt, bytes;
};

StageWs stage_layout(int64_t n, int64_t m, bool comp, bool classic)
{
    StageWs s;
    Carve cv;
    s.p = plan_sweep(n, n, m, true, comp, cv, !classic);
    s.nut = cv.take((size_t)n * sizeof(float));
    s.pos = cv.take((size_t)n * 16);
    s.str = cv.take((size_t)n * 16);
    s.dxdt = cv.take((size_t)n * 3 * sizeof(float));
    s.dGdt = cv.take((size_t)n * 3 * sizeof(float));
    s.bytes = cv.off;
    return s;
}

// The buffers vpm_step_tree adds after the treecode right-hand side's workspace.
size_t tree_step_extra(int64_t n)
{
    Carve cv;
    cv.take((size_t)n * 16);
    cv.take((size_t)n * 16);
    cv.take((size_t)n * 3 * sizeof(float));
    cv.take((size_t)n * 3 * sizeof(float));
    cv.take((size_t)n * 3 * sizeof(double));
    cv.take((size_t)n * 3 * sizeof(double));
    return cv.off + 256;  // room for aligning the first buffer after the right-hand side's
}

bool overflow_guard(const SweepPlan& p)
{
    // keep tot * B < 2^62 for the 64-bit stream-K arithmetic
    return (double)p.sk.tot * (double)p.sk.B < 4.0e18 && (double)p.sks.tot * (double)p.sks.B < 4.0e18;
}

vpm_status check_params(const vpm_params* prm)
{
    REQUIRE(prm != nullptr, "vpm_params is NULL");
    REQUIRE(prm->sigma > 0.f && isfinite(prm->sigma), "sigma must be finite and > 0 (got %g)", (double)prm->sigma);
    REQUIRE(prm->nu >= 0.f && isfinite(prm->nu), "nu must be finite and >= 0");
    REQUIRE(prm->c_v >= 0.f && isfinite(prm->c_v), "c_v must be finite and >= 0");
    REQUIRE(prm->seg_core >= 0.f && isfinite(prm->seg_core), "seg_core must be finite and >= 0");
    REQUIRE(prm->vatistas_n == 1 || prm->vatistas_n == 2, "vatistas_n must be 1 or 2 (got %d)", prm->vatistas_n);
    for (int a = 0; a < 3; ++a) REQUIRE(isfinite(prm->u_inf[a]), "u_inf must be finite");
    return VPM_OK;
}

}  // namespace

extern "C" {

const char* vpm_last_error(void) { return g_last_error.c_str(); }

int vpm_version(void) { return 10100; }

vpm_status vpm_device_error(int* code)
{
    REQUIRE(code != nullptr, "code is NULL");
    int* p = dev_err_ptr();
    if (!p) return fail(VPM_ERR_CUDA, "device error word unavailable");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "vpm_device_error");
    int v = 0;
    e = cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_device_error");
    const int z = 0;
    e = cudaMemcpy(p, &z, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_device_error");
    *code = (v & DEV_ERR_NONFINITE) ? VPM_ERR_NONFINITE : ((v & DEV_ERR_TIMEOUT) ? VPM_ERR_LIMIT : 0);
    return ok();
}

vpm_status vpm_workspace_size(int op, int64_t n_src, int64_t n_tgt, int64_t m_seg, int flags, size_t* bytes)
{
    REQUIRE(bytes != nullptr, "bytes is NULL");
    vpm_status s;
    if ((s = check_count(n_src, "n_src")) != VPM_OK) return s;
    if ((s = check_count(n_tgt, "n_tgt")) != VPM_OK) return s;
    if ((s = check_count(m_seg, "m_seg")) != VPM_OK) return s;
    const bool comp = flags & VPM_COMPENSATED;
    Carve cv;
    switch (op) {
    case VPM_OP_INDUCE: {
        Carve c2;
        const size_t a = plan_sweep(n_tgt, n_src, 0, true, comp, cv).bytes;
        const size_t b = plan_sweep(n_tgt, n_src, 0, false, comp, c2).bytes;
        *bytes = a > b ? a : b;
        break;
    }
    case VPM_OP_SEGMENTS: {
        Carve c2;
        const size_t a = plan_sweep(n_tgt, 0, m_seg, true, comp, cv).bytes;
        const size_t b = plan_sweep(n_tgt, 0, m_seg, false, comp, c2).bytes;
        *bytes = a > b ? a : b;
        break;
    }
    case VPM_OP_RHS:
        *bytes = plan_sweep(n_src, n_src, m_seg, true, comp, cv, !(flags & VPM_STRETCH_CLASSIC)).bytes +
                 rhs_extra(n_src);
        break;
    case VPM_OP_STEP:
        *bytes = step_layout(n_src, m_seg, comp, flags & VPM_STRETCH_CLASSIC).bytes;
        break;
    case VPM_OP_STAGE:
        *bytes = stage_layout(n_src, m_seg, comp, flags & VPM_STRETCH_CLASSIC).bytes;
        break;
    case VPM_OP_AIC_SOLVE:
        REQUIRE(n_tgt <= VPM_MAX_AIC, "AIC order %lld above %d", (long long)n_tgt, VPM_MAX_AIC);
        *bytes = aic_workspace((int)n_tgt);
        break;
    case VPM_OP_BACKWARD:
        *bytes = backward_workspace(n_src, n_tgt, comp);
        break;
    case VPM_OP_WAKE_CONVERT:
        *bytes = wake_workspace(n_src, false);
        break;
    case VPM_OP_LOADS:
        *bytes = loads_workspace(m_seg, n_tgt);
        break;
    case VPM_OP_WAKE_ROW:
        REQUIRE(n_src >= 1, "a wake row needs at least one panel");
        *bytes = wake_workspace(3 * n_src + 1, true);
        break;
    case VPM_OP_RHS_TREE:
    case VPM_OP_STEP_TREE: {
        TreeRhsWs r;
        const cudaError_t e = tree_rhs_layout(n_src, m_seg, r);
        if (e != cudaSuccess) return cuda_fail(e, "vpm_workspace_size: sort scratch query");
        *bytes = r.bytes + (op == VPM_OP_STEP_TREE ? tree_step_extra(n_src) : 0);
        break;
    }
    case VPM_OP_TREE: {
        const cudaError_t e = tree_workspace(n_src, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "vpm_workspace_size(VPM_OP_TREE): sort scratch query");
        break;
    }
    default:
        return fail(VPM_ERR_INVALID_ARG, "unknown op %d", op);
    }
    return ok();
}

vpm_status vpm_induce(const float* src_pos_d, const float* src_str_d, int64_t n_src, const float* tgt_d,
                      int64_t n_tgt, float sigma, int flags, float* u_d, float* grad_u_d, void* ws_d,
                      size_t ws_bytes, void* stream)
{
    vpm_status s;
    if ((s = check_count(n_src, "n_src")) != VPM_OK) return s;
    if ((s = check_count(n_tgt, "n_tgt")) != VPM_OK) return s;
    REQUIRE(sigma > 0.f && isfinite(sigma), "sigma must be finite and > 0 (got %g)", (double)sigma);
    if (n_tgt == 0) return ok();
    REQUIRE(tgt_d && aligned16(tgt_d), "tgt must be a 16-byte aligned device pointer");
    REQUIRE(u_d && aligned4(u_d), "u must be a 4-byte aligned device pointer");
    REQUIRE(!grad_u_d || aligned4(grad_u_d), "grad_u misaligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_src == 0) {
        cudaError_t e = cudaMemsetAsync(u_d, 0, sizeof(float) * 3 * (size_t)n_tgt, st);
        if (e == cudaSuccess && grad_u_d) e = cudaMemsetAsync(grad_u_d, 0, sizeof(float) * 9 * (size_t)n_tgt, st);
        return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_induce");
    }
    REQUIRE(src_pos_d && src_str_d && aligned16(src_pos_d) && aligned16(src_str_d),
            "src_pos/src_str must be 16-byte aligned device pointers");
    const bool comp = flags & VPM_COMPENSATED;
    Carve cv;
    const SweepPlan p = plan_sweep(n_tgt, n_src, 0, grad_u_d != nullptr, comp, cv);
    if (!overflow_guard(p)) return fail(VPM_ERR_LIMIT, "problem too large for the stream-K split");
    if (!ws_d || ws_bytes < p.bytes || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", p.bytes, ws_bytes);
    if (!dev_err_ptr()) return fail(VPM_ERR_CUDA, "no CUDA device");
    EpilogueOut o;
    o.mode = 0;
    o.u = u_d;
    o.grad_u = grad_u_d;
    o.check_finite = (flags & VPM_CHECK_FINITE) ? 1 : 0;
    cudaError_t e = run_sweep(p, static_cast<char*>(ws_d), tgt_d, src_pos_d, src_str_d, nullptr, nullptr, sigma, 0.f,
                              2, o, st);
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_induce");
}

vpm_status vpm_tree_induce(const float* pos_d, const float* str_d, int64_t n, float sigma, float theta, int order,
                           float* u_d, float* grad_u_d, void* ws_d, size_t ws_bytes, void* stream)
{
    vpm_status s;
    if ((s = check_count(n, "n")) != VPM_OK) return s;
    REQUIRE(sigma > 0.f && isfinite(sigma), "sigma must be finite and > 0 (got %g)", (double)sigma);
    REQUIRE(theta >= 0.f && theta <= 1.f, "theta must lie in [0, 1] (got %g)", (double)theta);
    REQUIRE(order >= 2 && order <= 4, "order must be 2, 3 or 4 (got %d)", order);
    if (n == 0) return ok();
    REQUIRE(pos_d && str_d && aligned16(pos_d) && aligned16(str_d), "pos/str must be 16-byte aligned device pointers");
    REQUIRE(u_d && aligned4(u_d), "u must be a 4-byte aligned device pointer");
    REQUIRE(!grad_u_d || aligned4(grad_u_d), "grad_u misaligned");
    size_t need = 0;
    const cudaError_t eq = tree_workspace(n, &need);
    if (eq != cudaSuccess) return cuda_fail(eq, "vpm_tree_induce: sort scratch query");
    if (!ws_d || ws_bytes < need || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", need, ws_bytes);
    if (!dev_err_ptr()) return fail(VPM_ERR_CUDA, "no CUDA device");
    cudaError_t e = run_tree_induce(pos_d, str_d, n, sigma, theta, order, u_d, grad_u_d, static_cast<char*>(ws_d),
                                    static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_tree_induce");
}

vpm_status vpm_segments_induce(const float* seg_a_d, const float* seg_b_d, int64_t m, const float* tgt_d,
                               int64_t n_tgt, float core, int vatistas_n, int flags, float* u_d, float* grad_u_d,
                               void* ws_d, size_t ws_bytes, void* stream)
{
    vpm_status s;
    if ((s = check_count(m, "m")) != VPM_OK) return s;
    if ((s = check_count(n_tgt, "n_tgt")) != VPM_OK) return s;
    REQUIRE(core >= 0.f && isfinite(core), "core must be finite and >= 0");
    REQUIRE(vatistas_n == 1 || vatistas_n == 2, "vatistas_n must be 1 or 2 (got %d)", vatistas_n);
    if (n_tgt == 0) return ok();
    REQUIRE(tgt_d && aligned16(tgt_d), "tgt must be a 16-byte aligned device pointer");
    REQUIRE(u_d && aligned4(u_d), "u must be a 4-byte aligned device pointer");
    REQUIRE(!grad_u_d || aligned4(grad_u_d), "grad_u misaligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (m == 0) {
        cudaError_t e = cudaMemsetAsync(u_d, 0, sizeof(float) * 3 * (size_t)n_tgt, st);
        if (e == cudaSuccess && grad_u_d) e = cudaMemsetAsync(grad_u_d, 0, sizeof(float) * 9 * (size_t)n_tgt, st);
        return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_segments_induce");
    }
    REQUIRE(seg_a_d && seg_b_d && aligned16(seg_a_d) && aligned16(seg_b_d),
            "seg_a/seg_b must be 16-byte aligned device pointers");
    const bool comp = flags & VPM_COMPENSATED;
    Carve cv;
    const SweepPlan p = plan_sweep(n_tgt, 0, m, grad_u_d != nullptr, comp, cv);
    if (!overflow_guard(p)) return fail(VPM_ERR_LIMIT, "problem too large for the stream-K split");
    if (!ws_d || ws_bytes < p.bytes || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", p.bytes, ws_bytes);
    if (!dev_err_ptr()) return fail(VPM_ERR_CUDA, "no CUDA device");
    EpilogueOut o;
    o.mode = 0;
    o.u = u_d;
    o.grad_u = grad_u_d;
    o.check_finite = (flags & VPM_CHECK_FINITE) ? 1 : 0;
    cudaError_t e = run_sweep(p, static_cast<char*>(ws_d), tgt_d, nullptr, nullptr, seg_a_d, seg_b_d, 1.f, core,
                              vatistas_n, o, st);
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_segments_induce");
}

static vpm_status rhs_into(const SweepPlan& p, char* ws, const float* pos, const float* str, int64_t n,
                           const float* seg_a, const float* seg_b, const vpm_params* prm, float* dxdt, float* dGdt,
                           float* nu_t, cudaStream_t st)
{
    EpilogueOut o;
    o.mode = 1;
    o.str = str;
    o.sigma = prm->sigma;
    o.c_v = prm->c_v;
    for (int a = 0; a < 3; ++a) o.uinf[a] = prm->u_inf[a];
    o.classic = (prm->flags & VPM_STRETCH_CLASSIC) ? 1 : 0;
    o.dxdt = dxdt;
    o.dGdt = dGdt;
    o.nu_t = nu_t;
    o.check_finite = (prm->flags & VPM_CHECK_FINITE) ? 1 : 0;
    cudaError_t e = run_sweep(p, ws, pos, pos, str, seg_a, seg_b, prm->sigma, prm->seg_core, prm->vatistas_n, o, st);
    if (e == cudaSuccess) e = run_pse(p, ws, pos, str, nu_t, (int)n, prm->sigma, prm->nu, dGdt, st);
    return e == cudaSuccess ? VPM_OK : cuda_fail(e, "vpm_rhs");
}

vpm_status vpm_rhs(const float* pos_d, const float* str_d, int64_t n, const float* seg_a_d, const float* seg_b_d,
                   int64_t m, const vpm_params* prm, float* dxdt_d, float* dGdt_d, float* nu_t_d, void* ws_d,
                   size_t ws_bytes, void* stream)
{
    vpm_status s;
    if ((s = check_params(prm)) != VPM_OK) return s;
    if ((s = check_count(n, "n")) != VPM_OK) return s;
    if ((s = check_count(m, "m")) != VPM_OK) return s;
    if (n == 0) return ok();
    REQUIRE(pos_d && str_d && aligned16(pos_d) && aligned16(str_d), "pos/str must be 16-byte aligned device pointers");
    REQUIRE(dxdt_d && dGdt_d && aligned4(dxdt_d) && aligned4(dGdt_d), "dxdt/dGdt must be device pointers");
    REQUIRE(m == 0 || (seg_a_d && seg_b_d && aligned16(seg_a_d) && aligned16(seg_b_d)),
            "seg_a/seg_b must be 16-byte aligned device pointers when m > 0");
    const bool comp = prm->flags & VPM_COMPENSATED;
    Carve cv;
    const SweepPlan p = plan_sweep(n, n, m, true, comp, cv, !(prm->flags & VPM_STRETCH_CLASSIC));
    const size_t off_nut = cv.take((size_t)n * sizeof(float));
    if (!overflow_guard(p)) return fail(VPM_ERR_LIMIT, "problem too large for the stream-K split");
    if (!ws_d || ws_bytes < cv.off || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", cv.off, ws_bytes);
    if (!dev_err_ptr()) return fail(VPM_ERR_CUDA, "no CUDA device");
    char* ws = static_cast<char*>(ws_d);
    float* nut = nu_t_d ? nu_t_d : reinterpret_cast<float*>(ws + off_nut);
    s = rhs_into(p, ws, pos_d, str_d, n, seg_a_d, seg_b_d, prm, dxdt_d, dGdt_d, nut, static_cast<cudaStream_t>(stream));
    return s == VPM_OK ? ok() : s;
}

vpm_status vpm_pack_state(const double* x_d, const double* G_d, const float* vol_d, int64_t n, float* pos_d,
                          float* str_d, void* stream)
{
    vpm_status s;
    if ((s = check_count(n, "n")) != VPM_OK) return s;
    if (n == 0) return ok();
    REQUIRE(x_d && G_d && vol_d && aligned8(x_d) && aligned8(G_d) && aligned4(vol_d),
            "x/G/vol must be aligned device pointers");
    REQUIRE(pos_d && str_d && aligned16(pos_d) && aligned16(str_d), "pos/str must be 16-byte aligned device pointers");
    cudaError_t e = run_cast_state(x_d, G_d, vol_d, (int)n, pos_d, str_d, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_pack_state");
}

vpm_status vpm_step(double* x_d, double* G_d, const float* vol_d, int64_t n, const float* seg_a_d,
                    const float* seg_b_d, int64_t m, const vpm_params* prm, double dt, void* ws_d, size_t ws_bytes,
                    void* stream)
{
    vpm_status s;
    if ((s = check_params(prm)) != VPM_OK) return s;
    if ((s = check_count(n, "n")) != VPM_OK) return s;
    if ((s = check_count(m, "m")) != VPM_OK) return s;
    REQUIRE(isfinite(dt), "dt must be finite");
    if (n == 0) return ok();
    REQUIRE(x_d && G_d && vol_d && aligned8(x_d) && aligned8(G_d) && aligned4(vol_d),
            "x/G/vol must be aligned device pointers");
    REQUIRE(m == 0 || (seg_a_d && seg_b_d && aligned16(seg_a_d) && aligned16(seg_b_d)),
            "seg_a/seg_b must be 16-byte aligned device pointers when m > 0");
    const bool comp = prm->flags & VPM_COMPENSATED;
    const StepWs L = step_layout(n, m, comp, prm->flags & VPM_STRETCH_CLASSIC);
    if (!overflow_guard(L.p)) return fail(VPM_ERR_LIMIT, "problem too large for the stream-K split");
    if (!ws_d || ws_bytes < L.bytes || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", L.bytes, ws_bytes);
    if (!dev_err_ptr()) return fail(VPM_ERR_CUDA, "no CUDA device");
    char* ws = static_cast<char*>(ws_d);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* nut = reinterpret_cast<float*>(ws + L.nut);
    float* pos = reinterpret_cast<float*>(ws + L.pos);
    float* str = reinterpret_cast<float*>(ws + L.str);
    float* dxdt = reinterpret_cast<float*>(ws + L.dxdt);
    float* dGdt = reinterpret_cast<float*>(ws + L.dGdt);
    double* qx = reinterpret_cast<double*>(ws + L.qx);
    double* qG = reinterpret_cast<double*>(ws + L.qG);
    cudaError_t e = run_cast_state(x_d, G_d, vol_d, (int)n, pos, str, st);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_step");
    for (int k = 0; k < 3; ++k) {
        s = rhs_into(L.p, ws, pos, str, n, seg_a_d, seg_b_d, prm, dxdt, dGdt, nut, st);
        if (s != VPM_OK) return s;
        e = run_rk3_stage(k, dt, x_d, G_d, qx, qG, dxdt, dGdt, vol_d, (int)n, k < 2 ? pos : nullptr,
                          k < 2 ? str : nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "vpm_step");
    }
    return ok();
}

vpm_status vpm_rk3_stage(int k, double* x_d, double* G_d, double* q_d, const float* vol_d, int64_t n,
                         const float* seg_a_d, const float* seg_b_d, int64_t m, const vpm_params* prm, double dt,
                         void* ws_d, size_t ws_bytes, void* stream)
{
    vpm_status s;
    if ((s = check_params(prm)) != VPM_OK) return s;
    if ((s = check_count(n, "n")) != VPM_OK) return s;
    if ((s = check_count(m, "m")) != VPM_OK) return s;
    REQUIRE(k >= 0 && k <= 2, "stage k must be 0, 1 or 2 (got %d)", k);
    REQUIRE(isfinite(dt), "dt must be finite");
    if (n == 0) return ok();
    REQUIRE(x_d && G_d && q_d && vol_d && aligned8(x_d) && aligned8(G_d) && aligned8(q_d) && aligned4(vol_d),
            "x/G/q/vol must be aligned device pointers");
    REQUIRE(m == 0 || (seg_a_d && seg_b_d && aligned16(seg_a_d) && aligned16(seg_b_d)),
            "seg_a/seg_b must be 16-byte aligned device pointers when m > 0");
    const bool comp = prm->flags & VPM_COMPENSATED;
    const StageWs L = stage_layout(n, m, comp, prm->flags & VPM_STRETCH_CLASSIC);
    if (!overflow_guard(L.p)) return fail(VPM_ERR_LIMIT, "problem too large for the stream-K split");
    if (!ws_d || ws_bytes < L.bytes || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", L.bytes, ws_bytes);
    if (!dev_err_ptr()) return fail(VPM_ERR_CUDA, "no CUDA device");
    char* ws = static_cast<char*>(ws_d);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* nut = reinterpret_cast<float*>(ws + L.nut);
    float* pos = reinterpret_cast<float*>(ws + L.pos);
    float* str = reinterpret_cast<float*>(ws + L.str);
    float* dxdt = reinterpret_cast<float*>(ws + L.dxdt);
    float* dGdt = reinterpret_cast<float*>(ws + L.dGdt);
    cudaError_t e = run_cast_state(x_d, G_d, vol_d, (int)n, pos, str, st);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_rk3_stage");
    s = rhs_into(L.p, ws, pos, str, n, seg_a_d, seg_b_d, prm, dxdt, dGdt, nut, st);
    if (s != VPM_OK) return s;
    e = run_rk3_stage(k, dt, x_d, G_d, q_d, q_d + 3 * (size_t)n, dxdt, dGdt, vol_d, (int)n, nullptr, nullptr, st);
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_rk3_stage");
}

vpm_status vpm_rhs_tree(const float* pos_d, const float* str_d, int64_t n, const float* seg_a_d, const float* seg_b_d,
                        int64_t m, const vpm_params* prm, float theta, int order, float* dxdt_d, float* dGdt_d,
                        float* nu_t_d, void* ws_d, size_t ws_bytes, void* stream)
{
    vpm_status s;
    if ((s = check_params(prm)) != VPM_OK) return s;
    if ((s = check_count(n, "n")) != VPM_OK) return s;
    if ((s = check_count(m, "m")) != VPM_OK) return s;
    REQUIRE(theta >= 0.f && theta <= 1.f, "theta must lie in [0, 1] (got %g)", (double)theta);
    REQUIRE(order >= 2 && order <= 4, "order must be 2, 3 or 4 (got %d)", order);
    if (n == 0) return ok();
    REQUIRE(pos_d && str_d && aligned16(pos_d) && aligned16(str_d), "pos/str must be 16-byte aligned device pointers");
    REQUIRE(dxdt_d && dGdt_d && aligned4(dxdt_d) && aligned4(dGdt_d), "dxdt/dGdt must be device pointers");
    REQUIRE(m == 0 || (seg_a_d && seg_b_d && aligned16(seg_a_d) && aligned16(seg_b_d)),
            "seg_a/seg_b must be 16-byte aligned device pointers when m > 0");
    TreeRhsWs r;
    cudaError_t e = tree_rhs_layout(n, m, r);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_rhs_tree: sort scratch query");
    if (!ws_d || ws_bytes < r.bytes || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", r.bytes, ws_bytes);
    if (!dev_err_ptr()) return fail(VPM_ERR_CUDA, "no CUDA device");
    e = run_tree_rhs(r, static_cast<char*>(ws_d), pos_d, str_d, n, seg_a_d, seg_b_d, m, prm, theta, order, dxdt_d,
                     dGdt_d, nu_t_d, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_rhs_tree");
}

vpm_status vpm_step_tree(double* x_d, double* G_d, const float* vol_d, int64_t n, const float* seg_a_d,
                         const float* seg_b_d, int64_t m, const vpm_params* prm, float theta, int order, double dt,
                         void* ws_d, size_t ws_bytes, void* stream)
{
    vpm_status s;
    if ((s = check_params(prm)) != VPM_OK) return s;
    if ((s = check_count(n, "n")) != VPM_OK) return s;
    if ((s = check_count(m, "m")) != VPM_OK) return s;
    REQUIRE(isfinite(dt), "dt must be finite");
    REQUIRE(theta >= 0.f && theta <= 1.f, "theta must lie in [0, 1] (got %g)", (double)theta);
    REQUIRE(order >= 2 && order <= 4, "order must be 2, 3 or 4 (got %d)", order);
    if (n == 0) return ok();
    REQUIRE(x_d && G_d && vol_d && aligned8(x_d) && aligned8(G_d) && aligned4(vol_d),
            "x/G/vol must be aligned device pointers");
    REQUIRE(m == 0 || (seg_a_d && seg_b_d && aligned16(seg_a_d) && aligned16(seg_b_d)),
            "seg_a/seg_b must be 16-byte aligned device pointers when m > 0");
    TreeRhsWs r;
    cudaError_t e = tree_rhs_layout(n, m, r);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_step_tree: sort scratch query");
    const size_t need = r.bytes + tree_step_extra(n);
    if (!ws_d || ws_bytes < need || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", need, ws_bytes);
    if (!dev_err_ptr()) return fail(VPM_ERR_CUDA, "no CUDA device");
    char* ws = static_cast<char*>(ws_d);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the step's own buffers after the right-hand side's
    Carve cv;
    cv.off = r.bytes;
    float* pos = reinterpret_cast<float*>(ws + cv.take((size_t)n * 16));
    float* str = reinterpret_cast<float*>(ws + cv.take((size_t)n * 16));
    float* dxdt = reinterpret_cast<float*>(ws + cv.take((size_t)n * 3 * sizeof(float)));
    float* dGdt = reinterpret_cast<float*>(ws + cv.take((size_t)n * 3 * sizeof(float)));
    double* qx = reinterpret_cast<double*>(ws + cv.take((size_t)n * 3 * sizeof(double)));
    double* qG = reinterpret_cast<double*>(ws + cv.take((size_t)n * 3 * sizeof(double)));
    e = run_cast_state(x_d, G_d, vol_d, (int)n, pos, str, st);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_step_tree");
    for (int k = 0; k < 3; ++k) {
        e = run_tree_rhs(r, ws, pos, str, n, seg_a_d, seg_b_d, m, prm, theta, order, dxdt, dGdt, nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "vpm_step_tree");
        e = run_rk3_stage(k, dt, x_d, G_d, qx, qG, dxdt, dGdt, vol_d, (int)n, k < 2 ? pos : nullptr,
                          k < 2 ? str : nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "vpm_step_tree");
    }
    return ok();
}

vpm_status aic_build(const float* rings_d, const float* colloc_d, const float* normal_d, int n, float core,
                     int vatistas_n, const float* v_rel_d, const float* w_ind_d, float* A_d, double* b_d,
                     void* stream)
{
    REQUIRE(n >= 0 && n <= VPM_MAX_AIC, "AIC order %d outside [0, %d]", n, VPM_MAX_AIC);
    REQUIRE(core >= 0.f && isfinite(core), "core must be finite and >= 0");
    REQUIRE(vatistas_n == 1 || vatistas_n == 2, "vatistas_n must be 1 or 2");
    if (n == 0) return ok();
    REQUIRE(rings_d && colloc_d && normal_d && aligned16(rings_d) && aligned16(colloc_d) && aligned16(normal_d),
            "rings/colloc/normal must be 16-byte aligned device pointers");
    REQUIRE(A_d && aligned4(A_d), "A must be a device pointer");
    REQUIRE(!b_d || (v_rel_d && aligned16(v_rel_d) && aligned8(b_d)), "b requires a 16-byte aligned v_rel");
    cudaError_t e = run_aic_build(rings_d, colloc_d, normal_d, n, core, vatistas_n, v_rel_d, w_ind_d, A_d, b_d,
                                  static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "aic_build");
}

vpm_status aic_solve(const float* A_d, const double* b_d, double* x_d, int n, double tol, int max_iter,
                     int* iters_out, double* berr_out, void* ws_d, size_t ws_bytes, void* stream)
{
    REQUIRE(n >= 0 && n <= VPM_MAX_AIC, "AIC order %d outside [0, %d]", n, VPM_MAX_AIC);
    REQUIRE(tol >= 0.0 && max_iter >= 0, "tol and max_iter must be >= 0");
    if (n == 0) return ok();
    REQUIRE(A_d && b_d && x_d && aligned4(A_d) && aligned8(b_d) && aligned8(x_d), "A/b/x must be device pointers");
    const size_t need = aic_workspace(n);
    if (!ws_d || ws_bytes < need || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", need, ws_bytes);
    const char* msg = "";
    vpm_status s = run_aic_solve(A_d, b_d, x_d, n, tol, max_iter, iters_out, berr_out, static_cast<char*>(ws_d),
                                 static_cast<cudaStream_t>(stream), &msg);
    if (s != VPM_OK) return fail(s, "%s", msg);
    return ok();
}

vpm_status vpm_induce_backward(const float* src_pos_d, const float* src_str_d, int64_t n_src, const float* tgt_d,
                               int64_t n_tgt, float sigma, int flags, const float* grad_out_d, float* dL_dx_d,
                               float* dL_dG_d, void* ws_d, size_t ws_bytes, void* stream)
{
    vpm_status s;
    if ((s = check_count(n_src, "n_src")) != VPM_OK) return s;
    if ((s = check_count(n_tgt, "n_tgt")) != VPM_OK) return s;
    REQUIRE(sigma > 0.f && isfinite(sigma), "sigma must be finite and > 0 (got %g)", (double)sigma);
    if (n_src == 0) return ok();
    REQUIRE(src_pos_d && src_str_d && aligned16(src_pos_d) && aligned16(src_str_d),
            "src_pos/src_str must be 16-byte aligned device pointers");
    REQUIRE(dL_dx_d && dL_dG_d && aligned4(dL_dx_d) && aligned4(dL_dG_d), "dL_dx/dL_dG must be device pointers");
    REQUIRE(n_tgt == 0 || (tgt_d && grad_out_d && aligned16(tgt_d) && aligned4(grad_out_d)),
            "tgt (16-byte aligned) and grad_out must be device pointers");
    const bool comp = flags & VPM_COMPENSATED;
    const size_t need = n_tgt > 0 ? backward_workspace(n_src, n_tgt, comp) : 0;
    if (n_tgt > 0 && (!ws_d || ws_bytes < need || !aligned16(ws_d)))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", need, ws_bytes);
    if (!dev_err_ptr()) return fail(VPM_ERR_CUDA, "no CUDA device");
    cudaError_t e = run_backward(static_cast<char*>(ws_d), ws_bytes, src_pos_d, src_str_d, (int)n_src, tgt_d,
                                 (int)n_tgt, sigma, comp, grad_out_d, dL_dx_d, dL_dG_d,
                                 static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_induce_backward");
}

vpm_status vpm_wake_convert(const double* edge_a_d, const double* edge_b_d, const double* gamma_d,
                            const double* gamma_nb_d, const int* has_nb_d, const int* trailed_d, int64_t m,
                            double ds_tip, int n_tip, int n_shed, double* x_d, double* G_d, int64_t ld_out,
                            int64_t* n_out, void* ws_d, size_t ws_bytes, void* stream)
{
    vpm_status s;
    if ((s = check_count(m, "m")) != VPM_OK) return s;
    if ((s = check_count(ld_out, "ld_out")) != VPM_OK) return s;
    REQUIRE(n_out != nullptr, "n_out is NULL");
    *n_out = 0;
    REQUIRE(ds_tip > 0.0 && isfinite(ds_tip), "ds_tip must be finite and > 0 (got %g)", ds_tip);
    REQUIRE(n_tip != 0 && n_shed >= 1, "n_tip must be nonzero and n_shed >= 1");
    if (m == 0) return ok();
    REQUIRE(edge_a_d && edge_b_d && gamma_d && trailed_d && aligned8(edge_a_d) && aligned8(edge_b_d) &&
                aligned8(gamma_d) && aligned4(trailed_d),
            "edge_a/edge_b/gamma/trailed must be device pointers");
    REQUIRE(!has_nb_d || (gamma_nb_d && aligned8(gamma_nb_d) && aligned4(has_nb_d)),
            "has_nb needs gamma_nb (device pointers)");
    REQUIRE(ld_out == 0 || (x_d && G_d && aligned8(x_d) && aligned8(G_d)), "x/G must be device pointers");
    const size_t need = wake_workspace(m, false);
    if (!ws_d || ws_bytes < need || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", need, ws_bytes);
    const char* msg = "";
    long long n = 0;
    s = run_wake_convert(edge_a_d, edge_b_d, gamma_d, gamma_nb_d, has_nb_d, trailed_d, m, ds_tip, n_tip, n_shed, x_d,
                         G_d, ld_out, &n, static_cast<char*>(ws_d), static_cast<cudaStream_t>(stream), &msg);
    *n_out = n;
    if (s != VPM_OK) return fail(s, "%s (%lld particles)", msg, n);
    return ok();
}

vpm_status vpm_wake_convert_row(const double* U_d, const double* D_d, const double* gamma_d, int64_t S, double ds_tip,
                                int n_tip, int n_shed, double* x_d, double* G_d, int64_t ld_out, int64_t* n_out,
                                void* ws_d, size_t ws_bytes, void* stream)
{
    vpm_status s;
    if ((s = check_count(S, "S")) != VPM_OK) return s;
    if ((s = check_count(ld_out, "ld_out")) != VPM_OK) return s;
    REQUIRE(n_out != nullptr, "n_out is NULL");
    *n_out = 0;
    REQUIRE(S >= 1, "a wake row needs at least one panel");
    REQUIRE(S <= (VPM_MAX_ITEMS - 1) / 3, "S = %lld gives more edges than %d", (long long)S, VPM_MAX_ITEMS);
    REQUIRE(ds_tip > 0.0 && isfinite(ds_tip), "ds_tip must be finite and > 0 (got %g)", ds_tip);
    REQUIRE(n_tip != 0 && n_shed >= 1, "n_tip must be nonzero and n_shed >= 1");
    REQUIRE(U_d && D_d && gamma_d && aligned8(U_d) && aligned8(D_d) && aligned8(gamma_d),
            "U/D/gamma must be device pointers");
    REQUIRE(ld_out == 0 || (x_d && G_d && aligned8(x_d) && aligned8(G_d)), "x/G must be device pointers");
    const size_t need = wake_workspace(3 * S + 1, true);
    if (!ws_d || ws_bytes < need || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", need, ws_bytes);
    const char* msg = "";
    long long n = 0;
    s = run_wake_convert_row(U_d, D_d, gamma_d, S, ds_tip, n_tip, n_shed, x_d, G_d, ld_out, &n,
                             static_cast<char*>(ws_d), static_cast<cudaStream_t>(stream), &msg);
    *n_out = n;
    if (s != VPM_OK) return fail(s, "%s (%lld particles)", msg, n);
    return ok();
}

vpm_status vpm_wake_segments(const double* nodes_d, const double* gamma_d, int64_t R, int64_t nb, int64_t S,
                             float* seg_a_d, float* seg_b_d, void* stream)
{
    REQUIRE(R >= 0 && nb >= 0 && S >= 0, "R, nb, S must be >= 0");
    REQUIRE(R * nb * S * 4 <= VPM_MAX_ITEMS, "more than %d segments", VPM_MAX_ITEMS);
    if (R * nb * S == 0) return ok();
    REQUIRE(nodes_d && gamma_d && aligned8(nodes_d) && aligned8(gamma_d), "nodes/gamma must be device pointers");
    REQUIRE(seg_a_d && seg_b_d && aligned16(seg_a_d) && aligned16(seg_b_d),
            "seg_a/seg_b must be 16-byte aligned device pointers");
    cudaError_t e = run_wake_segments(nodes_d, gamma_d, R, nb, S, seg_a_d, seg_b_d, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_wake_segments");
}

vpm_status vpm_ring_segments(const float* rings_d, const double* gamma_d, int64_t n, float* seg_a_d, float* seg_b_d,
                             void* stream)
{
    REQUIRE(n >= 0 && n <= VPM_MAX_ITEMS / 4, "ring count %lld outside [0, %d]", (long long)n, VPM_MAX_ITEMS / 4);
    if (n == 0) return ok();
    REQUIRE(rings_d && gamma_d && aligned16(rings_d) && aligned8(gamma_d), "rings/gamma must be device pointers");
    REQUIRE(seg_a_d && seg_b_d && aligned16(seg_a_d) && aligned16(seg_b_d),
            "seg_a/seg_b must be 16-byte aligned device pointers");
    cudaError_t e = run_ring_segments(rings_d, gamma_d, n, seg_a_d, seg_b_d, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_ring_segments");
}

vpm_status vpm_points_pack(const double* pts_d, int64_t n, float* tgt_d, void* stream)
{
    vpm_status s;
    if ((s = check_count(n, "n")) != VPM_OK) return s;
    if (n == 0) return ok();
    REQUIRE(pts_d && tgt_d && aligned8(pts_d) && aligned16(tgt_d), "pts/tgt must be device pointers (tgt 16-byte aligned)");
    cudaError_t e = run_points_pack(pts_d, n, tgt_d, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_points_pack");
}

vpm_status vpm_points_advect(double* pts_d, const float* u_d, int64_t n, double dt, const float* u_inf,
                             void* stream)
{
    vpm_status s;
    if ((s = check_count(n, "n")) != VPM_OK) return s;
    REQUIRE(isfinite(dt), "dt must be finite");
    if (n == 0) return ok();
    REQUIRE(pts_d && u_d && aligned8(pts_d) && aligned4(u_d), "pts/u must be device pointers");
    cudaError_t e = run_points_advect(pts_d, u_d, n, dt, u_inf, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_points_advect");
}

vpm_status vpm_segment_midpoints(const float* seg_a_d, const float* seg_b_d, int64_t m, float* tgt_d, void* stream)
{
    vpm_status s;
    if ((s = check_count(m, "m")) != VPM_OK) return s;
    if (m == 0) return ok();
    REQUIRE(seg_a_d && seg_b_d && tgt_d && aligned16(seg_a_d) && aligned16(seg_b_d) && aligned16(tgt_d),
            "seg_a/seg_b/tgt must be 16-byte aligned device pointers");
    cudaError_t e = run_segment_midpoints(seg_a_d, seg_b_d, m, tgt_d, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_segment_midpoints");
}

vpm_status vpm_blade_loads(const float* seg_a_d, const float* seg_b_d, int64_t m, const float* u_ind_d,
                           const double* omega, const double* hub, const double* u_inf, const float* rings_d,
                           const float* normal_d, const double* gamma_d, const double* gamma_prev_d, int64_t n,
                           double dt, double rho, double* out_d, void* ws_d, size_t ws_bytes, void* stream)
{
    vpm_status s;
    if ((s = check_count(m, "m")) != VPM_OK) return s;
    if ((s = check_count(n, "n")) != VPM_OK) return s;
    REQUIRE(omega && hub && u_inf, "omega, hub and u_inf are host double[3]");
    REQUIRE(out_d && aligned8(out_d), "out must be a device pointer to 6 doubles");
    REQUIRE(isfinite(rho) && (!gamma_prev_d || (dt > 0.0 && isfinite(dt))), "rho finite; dt > 0 with gamma_prev");
    REQUIRE(m == 0 || (seg_a_d && seg_b_d && u_ind_d && aligned16(seg_a_d) && aligned16(seg_b_d) && aligned4(u_ind_d)),
            "seg_a/seg_b (16-byte aligned) and u_ind must be device pointers");
    REQUIRE(!gamma_prev_d || n == 0 ||
                (rings_d && normal_d && gamma_d && aligned16(rings_d) && aligned16(normal_d) && aligned8(gamma_d) &&
                 aligned8(gamma_prev_d)),
            "rings/normal (16-byte aligned) and gamma must be device pointers");
    const size_t need = loads_workspace(m, n);
    if (!ws_d || ws_bytes < need || !aligned16(ws_d))
        return fail(VPM_ERR_WORKSPACE, "workspace needs %zu bytes (16-byte aligned), got %zu", need, ws_bytes);
    cudaError_t e = run_blade_loads(seg_a_d, seg_b_d, m, u_ind_d, omega, hub, u_inf, rings_d, normal_d, gamma_d,
                                    gamma_prev_d, gamma_prev_d ? n : 0, dt, rho, out_d, static_cast<char*>(ws_d),
                                    static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_blade_loads");
}

vpm_status vpm_selftest_wait(double limit_ms, int* completed, void* stream)
{
    REQUIRE(completed != nullptr, "completed is NULL");
    REQUIRE(limit_ms > 0.0 && limit_ms <= 2000.0, "limit_ms must be in (0, 2000] (got %g)", limit_ms);
    if (!dev_err_ptr()) return fail(VPM_ERR_CUDA, "no CUDA device");
    int h = -1;
    cudaError_t e = run_selftest_wait(limit_ms, &h, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "vpm_selftest_wait");
    *completed = h;
    return ok();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// vpm_induce_noalloc: vpm_induce for callers that cannot give the library a
// workspace because they have no way to allocate device memory themselves -- a
// solver written in C or Fortran that links this library without any CUDA memory
// manager, or a time-critical loop that is not allowed to allocate.  The scratch
// is a fixed array in the library's own device memory, reserved on every GPU that
// loads the library and kept until the process exits.  Its device address is
// looked up on every call, with the caller's device current; the first lookup on a
// device loads the library's module there.
// Nothing in it has to start at zero: each call writes every byte it later
// reads.  All calls share the one array, so calls whose GPU work overlaps race
// on it.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[VPM_NOALLOC_SCRATCH_BYTES];

// The array's device address on the current device, looked up on every call (a
// cheap query once the module is loaded), so that it is never stale.
cudaError_t noalloc_scratch_address(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" vpm_status vpm_induce_noalloc(const float* src_pos_d, const float* src_str_d, int64_t n_src,
                                         const float* tgt_d, int64_t n_tgt, float sigma, int flags, float* u_d,
                                         float* grad_u_d, void* stream)
{
    vpm_status s;
    if ((s = check_count(n_src, "n_src")) != VPM_OK) return s;
    if ((s = check_count(n_tgt, "n_tgt")) != VPM_OK) return s;
    REQUIRE(sigma > 0.f && isfinite(sigma), "sigma must be finite and > 0 (got %g)", (double)sigma);
    if (n_tgt == 0) return ok();
    REQUIRE(tgt_d && aligned16(tgt_d), "tgt must be a 16-byte aligned device pointer");
    REQUIRE(u_d && aligned4(u_d), "u must be a 4-byte aligned device pointer");
    REQUIRE(!grad_u_d || aligned4(grad_u_d), "grad_u misaligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_src == 0) {
        cudaError_t e = cudaMemsetAsync(u_d, 0, sizeof(float) * 3 * (size_t)n_tgt, st);
        if (e == cudaSuccess && grad_u_d) e = cudaMemsetAsync(grad_u_d, 0, sizeof(float) * 9 * (size_t)n_tgt, st);
        return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_induce_noalloc");
    }
    REQUIRE(src_pos_d && src_str_d && aligned16(src_pos_d) && aligned16(src_str_d),
            "src_pos/src_str must be 16-byte aligned device pointers");
    const bool comp = flags & VPM_COMPENSATED;
    Carve cv;
    const SweepPlan p = plan_sweep(n_tgt, n_src, 0, grad_u_d != nullptr, comp, cv);
    if (!overflow_guard(p)) return fail(VPM_ERR_LIMIT, "problem too large for the stream-K split");
    if (p.bytes > (size_t)VPM_NOALLOC_SCRATCH_BYTES)
        return fail(VPM_ERR_LIMIT,
                    "vpm_induce_noalloc: %lld sources onto %lld targets need %zu bytes of scratch, more than the "
                    "%d bytes reserved; use vpm_induce with a workspace",
                    (long long)n_src, (long long)n_tgt, p.bytes, VPM_NOALLOC_SCRATCH_BYTES);
    if (!dev_err_ptr()) return fail(VPM_ERR_CUDA, "no CUDA device");
    void* ws = nullptr;
    cudaError_t e = noalloc_scratch_address(&ws);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_induce_noalloc: scratch address");
    EpilogueOut o;
    o.mode = 0;
    o.u = u_d;
    o.grad_u = grad_u_d;
    o.check_finite = (flags & VPM_CHECK_FINITE) ? 1 : 0;
    e = run_sweep(p, static_cast<char*>(ws), tgt_d, src_pos_d, src_str_d, nullptr, nullptr, sigma, 0.f, 2, o, st);
    return e == cudaSuccess ? ok() : cuda_fail(e, "vpm_induce_noalloc");
}
