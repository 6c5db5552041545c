// lbm_api.cu -- host side of the C ABI declared in include/lbm.h.
//
// Validates parameters, lays out the caller-owned workspace, derives the
// kernel constants from the physical parameters and enqueues the kernels on
// the caller's stream.  The library allocates no device memory.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include "lbm_internal.h"

using namespace lbmgpu;

namespace {
// A named NVTX range over an entry point, for profilers (ncu --nvtx); inert
// when no tool is attached.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};
}  // namespace

struct lbm_ctx {
    lbm_params p;
    KParams kp;
    Views v;
    cudaStream_t stream;
    int64_t step;
    int odd;          // parity of the AA layout: the next step is odd when set
    char err[256];
};

namespace {

thread_local char g_err[256] = "";

constexpr size_t ALIGN = 256;
inline size_t up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    size_t f, phi, stage, chibar, colmax, part, fwpart, ddiag, fgrad, total;
    unsigned nblocks;
};

int q_of(const lbm_params* p) { return p->model == LBM_CUMULANT_Q27 ? 27 : 19; }
int ns_of(const lbm_params* p) {
    return p->scalar == LBM_SCALAR_Q6 ? 6 : (p->scalar == LBM_SCALAR_Q27 ? 27 : 7);
}
Kind kind(const lbm_params* p) { return Kind{p->model, p->scalar, p->storage}; }
size_t elem_size(const lbm_params* p) { return p->storage == LBM_FP32 ? 4 : 2; }

bool finite(double v) { return isfinite(v) != 0; }

const char* check(const lbm_params* p) {
    if (!p) return "params is NULL";
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return "nx, ny, nz must be >= 1";
    if (p->ny > 65535 || p->nz > 65535) return "ny and nz must be <= 65535";
    if ((double)p->nx * p->ny * p->nz >= 2147483648.0) return "nx*ny*nz must be < 2^31";
    if (p->model != LBM_BGK_SMAG_Q19 && p->model != LBM_CUMULANT_Q27) return "unknown model";
    if (p->scalar != LBM_SCALAR_Q7 && p->scalar != LBM_SCALAR_Q6 && p->scalar != LBM_SCALAR_Q27)
        return "unknown scalar lattice";
    if (p->model == LBM_BGK_SMAG_Q19 && p->scalar == LBM_SCALAR_Q27)
        return "the D3Q27 scalar runs with the cumulant model";
    if (p->model == LBM_CUMULANT_Q27 && p->scalar == LBM_SCALAR_Q6)
        return "the D3Q6 scalar runs with the BGK model";
    if (p->storage != LBM_FP32 && p->storage != LBM_FP16S && p->storage != LBM_BF16S)
        return "unknown storage";
    if (p->flags & ~(LBM_FLAG_NO_COLLIDE | LBM_FLAG_PERIODIC_X | LBM_FLAG_PERIODIC_Z |
                     LBM_FLAG_ONE_NODE | LBM_FLAG_TMA_STAGED | LBM_FLAG_TEST_STALL |
                     LBM_FLAG_TEST_BOUNDS))
        return "unknown flag bits";
    if ((p->flags & LBM_FLAG_TEST_BOUNDS) && !lbm_debug_build())
        return "LBM_FLAG_TEST_BOUNDS needs the debug build (liblbm_debug.so)";
    if (!finite(p->nu) || p->nu <= 0.0) return "nu must be finite and > 0";
    if (!finite(p->D) || p->D <= 0.0) return "D must be finite and > 0";
    if (!finite(p->cs_smag) || p->cs_smag < 0.0) return "cs_smag must be finite and >= 0";
    if (!finite(p->sc_t) || p->sc_t <= 0.0) return "sc_t must be finite and > 0";
    if (!finite(p->gprime)) return "gprime must be finite";
    if (!finite(p->eg[0]) || !finite(p->eg[1]) || !finite(p->eg[2])) return "eg must be finite";
    if (p->model == LBM_CUMULANT_Q27 && (!finite(p->omega_bulk) || p->omega_bulk <= 0.0 ||
                                         p->omega_bulk >= 2.0))
        return "omega_bulk must lie in (0, 2)";
    if (p->nx_global != 0 && p->nx_global < p->nx) return "nx_global must be 0 or >= nx";
    if (p->x_offset < 0 || (double)p->x_offset + p->nx > (p->nx_global ? p->nx_global : p->nx))
        return "x_offset + nx must not exceed nx_global";
    if (p->nx_global > p->nx && (p->flags & LBM_FLAG_PERIODIC_X))
        return "an x-slab takes no LBM_FLAG_PERIODIC_X (its x ends are slab faces)";
    if (p->x0 < 0 || p->x0 > (p->nx_global ? p->nx_global : p->nx))
        return "x0 must lie in [0, nx_global]";
    if (p->H <= 0) return "H must be > 0";
    if (!finite(p->noise_amp) || p->noise_amp < 0.0) return "noise_amp must be finite and >= 0";
    if (!finite(p->front_threshold)) return "front_threshold must be finite";
    if (!finite(p->scale_f) || p->scale_f <= 0.0 || !finite(p->scale_phi) || p->scale_phi <= 0.0)
        return "scale_f and scale_phi must be finite and > 0";
    return nullptr;
}

Layout layout(const lbm_params* p) {
    Layout L;
    const size_t N = (size_t)p->nx * p->ny * p->nz, es = elem_size(p);
    L.nblocks = diag_block_count(p->nx, p->nz);
    size_t o = 0;
    L.f = o;      o = up(o + (size_t)q_of(p) * N * es);
    L.phi = o;    o = up(o + (size_t)ns_of(p) * N * es);
    // 16-bit storage: the scalar's rest population in an FP32 row after the
    // 16-bit rows (rest_row in lbm_common.cuh; none on D3Q6)
    if (es == 2 && p->scalar != LBM_SCALAR_Q6) o = up(o + N * sizeof(float));
    L.stage = o;  o = up(o + N * sizeof(float));
    L.chibar = o; o = up(o + (size_t)p->nx * p->nz * sizeof(float));
    L.colmax = o; o = up(o + (size_t)p->nx * sizeof(unsigned));
    L.part = o;   o = up(o + (size_t)L.nblocks * 2 * sizeof(double));
    L.fwpart = o; o = up(o + (size_t)L.nblocks * 2 * sizeof(float));
    // the diagnostics record, the two device flag words and the debug
    // build's index-check record (DbgRecord, lbm_common.cuh)
    L.ddiag = o;  o = up(o + sizeof(DevDiag) + 2 * sizeof(int) + sizeof(DbgRecord));
    L.fgrad = o;  o = up(o + sizeof(FrontGrad));
    L.total = o;
    return L;
}

KParams kparams(const lbm_params* p) {
    KParams k;
    memset(&k, 0, sizeof k);
    k.nx = p->nx; k.ny = p->ny; k.nz = p->nz; k.flags = p->flags;
    k.N = (unsigned)((size_t)p->nx * p->ny * p->nz);
    k.nxny = (unsigned)((size_t)p->nx * p->ny);
    const double tau0 = 3.0 * p->nu + 0.5;                        // Eq. 25
    k.tau0 = (float)tau0;
    k.A = (float)(18.0 * sqrt(2.0) * p->cs_smag * p->cs_smag);    // Eq. 34, R3
    // D = c_s^2 (tau_Phi - 1/2) (Eq. 30): c_s^2 = 1/4 on D3Q7, 1/3 on D3Q6
    const double cs2 = p->scalar == LBM_SCALAR_Q6 ? 1.0 / 3.0 : 0.25;
    k.taup0 = (float)(0.5 + p->D / cs2);
    // tau_Phi = taup0 + (nu_T / Sc_T) / c_s^2, nu_T = (tau - tau0) / 3 (Eq. 35)
    k.kT = p->model == LBM_BGK_SMAG_Q19 ? (float)(1.0 / (3.0 * p->sc_t * cs2)) : 0.0f;
    k.omD = (float)(1.0 / (3.0 * p->D + 0.5));                    // Eq. 51
    k.om1 = (float)(1.0 / tau0);                                  // Eq. 58
    k.om2 = (float)p->omega_bulk;
    k.gx = (float)(p->gprime * p->eg[0]);                         // Eq. 11
    k.gy = (float)(p->gprime * p->eg[1]);
    k.gz = (float)(p->gprime * p->eg[2]);
    const bool s16 = p->storage != LBM_FP32;
    k.sf = s16 ? (float)p->scale_f : 1.0f;
    k.isf = 1.0f / k.sf;
    k.sp = s16 ? (float)p->scale_phi : 1.0f;
    k.isp = 1.0f / k.sp;
    // 16-bit storage holds the scalar as scale_phi (Phi - chi_s w)
    k.chi_s = s16 ? (float)LBM_SCALAR_CHI16 : 1.0f;
    k.nu = (float)p->nu;
    // the correctly rounded FP32 quotient, bit-identical to 1.0f / taup0 on
    // the device, so that a kernel may take either form
    k.omp0 = 1.0f / k.taup0;
    // 64-bit element offsets in the step kernels once (Q + NS) N reaches 2^32
    k.wide = (double)(q_of(p) + ns_of(p)) * k.N >= 4294967296.0 ? 1 : 0;
    k.x_off = p->x_offset;
    k.nxg = p->nx_global ? p->nx_global : p->nx;
    return k;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
    snprintf(c->err, sizeof c->err, "%s: %s", where, cudaGetErrorString(e));
    return LBM_ERR_CUDA;
}

lbm_status arg_fail(lbm_ctx* c, const char* what) {
    if (c) snprintf(c->err, sizeof c->err, "%s", what);
    else snprintf(g_err, sizeof g_err, "%s", what);
    return LBM_ERR_ARG;
}

// The saved steps and the adjoint kernels use 32-bit element offsets of the
// canonical layout: boxes with (Q + NS) N < 2^32.
lbm_status narrow_check(lbm_ctx* c) {
    if (c->kp.wide) {
        snprintf(c->err, sizeof c->err,
                 "saved steps and the adjoint need (Q + NS) * nx * ny * nz < 2^32");
        return LBM_ERR_STATE;
    }
    return LBM_OK;
}

}  // namespace

namespace lbmgpu {
// Message returned by lbm_last_error(NULL) on this thread.
void lbm_set_thread_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace lbmgpu

extern "C" {

const char* lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_ERR_ARG: return "invalid argument";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_NOMEM: return "workspace too small";
        case LBM_ERR_UNSTABLE: return "unstable: non-finite value or rho <= 0";
        case LBM_ERR_STATE: return "call not valid in this state";
        case LBM_ERR_TIMEOUT: return "timeout";
        case LBM_ERR_BOUNDS: return "index check failed (debug build)";
    }
    return "unknown status";
}

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err : g_err; }

lbm_status lbm_validate(const lbm_params* p) {
    const char* m = check(p);
    if (m) { snprintf(g_err, sizeof g_err, "%s", m); return LBM_ERR_ARG; }
    return LBM_OK;
}

size_t lbm_workspace_bytes(const lbm_params* p) {
    if (check(p)) return 0;
    return layout(p).total;
}

lbm_status lbm_init(const lbm_params* p, void* workspace, size_t bytes, void* cuda_stream,
                    lbm_ctx** out) {
    const Range range("lbm_init");
    if (!out) return arg_fail(nullptr, "out is NULL");
    const char* m = check(p);
    if (m) return arg_fail(nullptr, m);
    if (!workspace) return arg_fail(nullptr, "workspace is NULL");
    if ((uintptr_t)workspace % ALIGN) return arg_fail(nullptr, "workspace must be 256-byte aligned");
    const Layout L = layout(p);
    if (bytes < L.total) {
        snprintf(g_err, sizeof g_err, "workspace has %zu bytes, needs %zu", bytes, L.total);
        return LBM_ERR_NOMEM;
    }
    lbm_ctx* c = (lbm_ctx*)calloc(1, sizeof(lbm_ctx));
    if (!c) return arg_fail(nullptr, "host allocation of the context failed");
    c->p = *p;
    c->kp = kparams(p);
    c->stream = (cudaStream_t)cuda_stream;
    uint8_t* w = (uint8_t*)workspace;
    c->v.f = w + L.f;
    c->v.phi = w + L.phi;
    c->v.stage = (float*)(w + L.stage);
    c->v.chibar = (float*)(w + L.chibar);
    c->v.colmax = (unsigned*)(w + L.colmax);
    c->v.part = (double*)(w + L.part);
    c->v.fwpart = (float*)(w + L.fwpart);
    c->v.ddiag = (DevDiag*)(w + L.ddiag);
    c->v.devflags = (int*)(w + L.ddiag + sizeof(DevDiag));
    c->v.fgrad = (FrontGrad*)(w + L.fgrad);
    c->v.diag_blocks = L.nblocks;
    c->kp.devflags = c->v.devflags;
    cudaError_t e = launch_init(c->kp, kind(p), c->v, nullptr, p->x0, p->noise_amp,
                                p->seed, c->stream);
    if (e != cudaSuccess) {
        snprintf(g_err, sizeof g_err, "init launch: %s", cudaGetErrorString(e));
        free(c);
        return LBM_ERR_CUDA;
    }
    c->step = 0;
    c->odd = 0;
    *out = c;
    return LBM_OK;
}

lbm_status lbm_set_scalar(lbm_ctx* c, const float* chi0) {
    const Range range("lbm_set_scalar");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (!chi0) return arg_fail(c, "chi0 is NULL");
    cudaError_t e = cudaMemcpyAsync(c->v.stage, chi0, (size_t)c->kp.N * sizeof(float),
                                    cudaMemcpyDefault, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_scalar copy");
    e = launch_init(c->kp, kind(&c->p), c->v, c->v.stage, 0, 0.0, 0, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_scalar init");
    c->step = 0;
    c->odd = 0;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int32_t nsteps) {
    const Range range("lbm_step");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (nsteps < 0) return arg_fail(c, "nsteps must be >= 0");
    for (int32_t s = 0; s < nsteps; ++s) {
        cudaError_t e = launch_step(c->kp, kind(&c->p), c->odd != 0, c->v.f, c->v.phi,
                                    nullptr, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
        c->odd ^= 1;
        ++c->step;
    }
    return LBM_OK;
}

lbm_status lbm_step_save(lbm_ctx* c, float* state_out) {
    const Range range("lbm_step_save");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (!state_out) return arg_fail(c, "state_out is NULL");
    if (lbm_status s = narrow_check(c); s != LBM_OK) return s;
    cudaError_t e = launch_step(c->kp, kind(&c->p), c->odd != 0, c->v.f, c->v.phi,
                                state_out, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
    c->odd ^= 1;
    ++c->step;
    return LBM_OK;
}

lbm_status lbm_macros(lbm_ctx* c, float* rho, float* u, float* chi) {
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (!rho && !u && !chi) return LBM_OK;
    cudaError_t e = launch_macros(c->kp, kind(&c->p), c->odd != 0, c->v, rho, u, chi,
                                  c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "macros launch");
    return LBM_OK;
}

lbm_status lbm_diag(lbm_ctx* c, lbm_diagnostics* out) {
    const Range range("lbm_diag");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (!out) return arg_fail(c, "out is NULL");
    cudaError_t e = launch_diag(c->kp, kind(&c->p), c->odd != 0, c->v,
                                c->p.front_threshold, c->p.x0, (double)c->p.H, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "diag launch");
    struct { DevDiag d; int flags[2]; } rec;
    e = cudaMemcpyAsync(&rec, c->v.ddiag, sizeof rec, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "diag copy");
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "diag sync");
    out->front = rec.d.front;
    out->front_node = rec.d.front_node;
    out->Fw = rec.d.Fw;
    out->mass_delta = rec.d.mass_delta;
    out->scalar_mass = rec.d.scalar_mass;
    out->step = c->step;
    out->flags = rec.flags[0];
    out->pad_ = 0;
    if (rec.flags[0]) {
        snprintf(c->err, sizeof c->err, "sticky device flags 0x%x", rec.flags[0]);
        if (rec.flags[0] & LBM_DEVFLAG_BOUNDS) return LBM_ERR_BOUNDS;
        return (rec.flags[0] & LBM_DEVFLAG_TIMEOUT) ? LBM_ERR_TIMEOUT : LBM_ERR_UNSTABLE;
    }
    return LBM_OK;
}

lbm_status lbm_fw_accumulate(lbm_ctx* c, double* acc_dev, double weight) {
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (!acc_dev) return arg_fail(c, "acc_dev is NULL");
    if (!isfinite(weight)) return arg_fail(c, "weight must be finite");
    cudaError_t e = launch_fw_accumulate(c->kp, kind(&c->p), c->odd != 0, c->v,
                                         acc_dev, weight, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "fw launch");
    return LBM_OK;
}

lbm_status lbm_get_state(lbm_ctx* c, float* dst) {
    const Range range("lbm_get_state");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (!dst) return arg_fail(c, "dst is NULL");
    cudaError_t e = launch_get_state(c->kp, kind(&c->p), c->odd != 0, c->v, dst,
                                     c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_state launch");
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx* c, const float* src, int64_t step) {
    const Range range("lbm_set_state");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (!src) return arg_fail(c, "src is NULL");
    if (step < 0) return arg_fail(c, "step must be >= 0");
    cudaError_t e = launch_set_state(c->kp, kind(&c->p), c->v, src, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_state launch");
    c->step = step;
    c->odd = 0;
    return LBM_OK;
}

namespace {
// One reverse step of the model's adjoint (BGK: with the C_s term).
cudaError_t adjoint_step_any(lbm_ctx* c, const float* state, const float* lam_next, float* lam,
                             double* dcs, float wfw, cudaStream_t st) {
    if (c->p.model == LBM_CUMULANT_Q27)
        return launch_cumulant_adjoint_step(c->kp, state, lam_next, lam, wfw, st);
    const float dAdCs = (float)(36.0 * sqrt(2.0) * c->p.cs_smag);
    return launch_adjoint_step(c->kp, state, lam_next, lam, dcs, wfw, dAdCs, st);
}

cudaError_t push_step_any(lbm_ctx* c, const float* src, float* dst, cudaStream_t st) {
    if (c->p.model == LBM_CUMULANT_Q27) return launch_cumulant_push_step(c->kp, src, dst, st);
    return launch_push_step(c->kp, src, dst, st);
}

cudaStream_t stream_or_ctx(lbm_ctx* c, void* stream) {
    return stream ? (cudaStream_t)stream : c->stream;
}

lbm_status sweep_check(lbm_ctx* c) {
    if (lbm_status s = narrow_check(c); s != LBM_OK) return s;
    if (c->p.storage != LBM_FP32 || c->p.scalar != LBM_SCALAR_Q7) {
        snprintf(c->err, sizeof c->err,
                 "the adjoint sweep exists for the D3Q7 scalar and FP32 storage");
        return LBM_ERR_STATE;
    }
    return LBM_OK;
}

lbm_status adjoint_model_check(lbm_ctx* c) {
    if (lbm_status s = narrow_check(c); s != LBM_OK) return s;
    if (c->p.scalar != LBM_SCALAR_Q7) {
        snprintf(c->err, sizeof c->err, "the adjoint exists for the D3Q7 scalar");
        return LBM_ERR_STATE;
    }
    return LBM_OK;
}
}  // namespace

lbm_status lbm_adjoint_step(lbm_ctx* c, const float* state_n, const float* lam_next, float* lam_n,
                            double* dJdCs_dev, double w_fw) {
    const Range range("lbm_adjoint_step");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (lbm_status s = adjoint_model_check(c); s != LBM_OK) return s;
    if (!state_n || !lam_n) return arg_fail(c, "state_n and lam_n must not be NULL");
    if (lam_n == lam_next || lam_n == state_n) return arg_fail(c, "lam_n must not alias its inputs");
    if (!isfinite(w_fw)) return arg_fail(c, "w_fw must be finite");
    cudaError_t e = adjoint_step_any(c, state_n, lam_next, lam_n, dJdCs_dev, (float)w_fw, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint launch");
    return LBM_OK;
}

lbm_status lbm_objective_forward(lbm_ctx* c, int32_t nsteps, int32_t K, float* ckpt,
                                 double* J_dev) {
    const Range range("lbm_objective_forward");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (nsteps < 0 || K < 1) return arg_fail(c, "nsteps must be >= 0 and K >= 1");
    const size_t S = (size_t)(q_of(&c->p) + ns_of(&c->p)) * c->kp.N;
    for (int32_t n = 0; n < nsteps; ++n) {
        cudaError_t e = cudaSuccess;
        if (ckpt && n % K == 0)
            e = launch_get_state(c->kp, kind(&c->p), c->odd != 0, c->v,
                                 ckpt + (size_t)(n / K) * S, c->stream);
        if (e == cudaSuccess)
            e = launch_step(c->kp, kind(&c->p), c->odd != 0, c->v.f, c->v.phi,
                            nullptr, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "objective forward launch");
        c->odd ^= 1;
        ++c->step;
        if (J_dev)
            e = launch_fw_accumulate(c->kp, kind(&c->p), c->odd != 0, c->v, J_dev, 1.0,
                                     c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "objective forward launch");
    }
    return LBM_OK;
}

lbm_status lbm_recompute_segment(lbm_ctx* c, const float* ckpt, int32_t k, float* seg,
                                 void* stream) {
    const Range range("lbm_recompute_segment");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (lbm_status s = sweep_check(c); s != LBM_OK) return s;
    if (k < 1) return arg_fail(c, "k must be >= 1");
    if (!ckpt || (k > 1 && !seg)) return arg_fail(c, "NULL buffer");
    const size_t S = (size_t)(q_of(&c->p) + ns_of(&c->p)) * c->kp.N;
    const cudaStream_t st = stream_or_ctx(c, stream);
    cudaError_t e = cudaSuccess;
    // s_{n0+1} .. s_{n0+k-1} into seg[1 .. k-1]
    const float* prev = ckpt;
    for (int32_t j = 1; j < k && e == cudaSuccess; ++j) {
        e = push_step_any(c, prev, seg + (size_t)j * S, st);
        prev = seg + (size_t)j * S;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "recompute segment");
    return LBM_OK;
}

lbm_status lbm_adjoint_sweep(lbm_ctx* c, const float* ckpt, const float* seg, int64_t n0,
                             int32_t k, float* lam, float* tmp, double* dJdCs_dev, double w_fw,
                             void* stream) {
    const Range range("lbm_adjoint_sweep");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (lbm_status s = sweep_check(c); s != LBM_OK) return s;
    if (k < 1 || n0 < 0) return arg_fail(c, "k must be >= 1 and n0 >= 0");
    if (!ckpt || !lam || !tmp || (k > 1 && !seg)) return arg_fail(c, "NULL buffer");
    if (lam == tmp) return arg_fail(c, "lam and tmp must differ");
    if (!isfinite(w_fw)) return arg_fail(c, "w_fw must be finite");
    const size_t S = (size_t)(q_of(&c->p) + ns_of(&c->p)) * c->kp.N;
    const cudaStream_t st = stream_or_ctx(c, stream);
    cudaError_t e = cudaSuccess;
    // lam_{n0+k} -> lam_{n0}
    float* cur = lam;
    float* nxt = tmp;
    for (int32_t j = k - 1; j >= 0 && e == cudaSuccess; --j) {
        const int64_t n = n0 + j;
        const float* sn = j == 0 ? ckpt : seg + (size_t)j * S;
        e = adjoint_step_any(c, sn, cur, nxt, dJdCs_dev, n >= 1 ? (float)w_fw : 0.0f, st);
        float* t = cur; cur = nxt; nxt = t;
    }
    if (e == cudaSuccess && cur != lam)
        e = cudaMemcpyAsync(lam, cur, S * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint sweep");
    return LBM_OK;
}

lbm_status lbm_adjoint_segment(lbm_ctx* c, const float* ckpt, int64_t n0, int32_t k, float* seg,
                               float* lam, float* tmp, double* dJdCs_dev, double w_fw) {
    const Range range("lbm_adjoint_segment");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (k < 1 || n0 < 0) return arg_fail(c, "k must be >= 1 and n0 >= 0");
    lbm_status s = lbm_recompute_segment(c, ckpt, k, seg, nullptr);
    if (s != LBM_OK) return s;
    return lbm_adjoint_sweep(c, ckpt, seg, n0, k, lam, tmp, dJdCs_dev, w_fw, nullptr);
}

lbm_status lbm_front_adjoint(lbm_ctx* c, const float* state, float* lam, double* front_dev) {
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (!state) return arg_fail(c, "state is NULL");
    if (lam == state) return arg_fail(c, "lam must not alias state");
    cudaError_t e = launch_front_adjoint(c->kp, q_of(&c->p), ns_of(&c->p), c->v, state, lam,
                                         front_dev, c->p.front_threshold, c->p.x0,
                                         (double)c->p.H, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "front_adjoint launch");
    return LBM_OK;
}

lbm_status lbm_adjoint_chi0(lbm_ctx* c, const float* lam0, float* grad_chi0) {
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (!lam0 || !grad_chi0) return arg_fail(c, "lam0 and grad_chi0 must not be NULL");
    if (lbm_status s = adjoint_model_check(c); s != LBM_OK) return s;
    cudaError_t e = launch_adjoint_chi0(c->kp, q_of(&c->p), lam0, grad_chi0, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint_chi0 launch");
    return LBM_OK;
}

size_t lbm_halo_bytes(const lbm_params* p) {
    if (check(p)) return 0;
    return halo_elems(q_of(p), ns_of(p), p->ny, p->nz) * elem_size(p);
}

lbm_status lbm_halo_pack(lbm_ctx* c, int32_t face, void* buf) {
    const Range range("lbm_halo_pack");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (face != 0 && face != 1) return arg_fail(c, "face must be 0 (x = 0) or 1 (x = nx - 1)");
    if (!buf) return arg_fail(c, "buf is NULL");
    cudaError_t e = launch_halo(c->kp, kind(&c->p), face, true, c->v.f, c->v.phi, buf, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "halo_pack launch");
    return LBM_OK;
}

lbm_status lbm_halo_unpack(lbm_ctx* c, int32_t face, const void* buf) {
    const Range range("lbm_halo_unpack");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (face != 0 && face != 1) return arg_fail(c, "face must be 0 (x = 0) or 1 (x = nx - 1)");
    if (!buf) return arg_fail(c, "buf is NULL");
    cudaError_t e = launch_halo(c->kp, kind(&c->p), face, false, c->v.f, c->v.phi,
                                const_cast<void*>(buf), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "halo_unpack launch");
    return LBM_OK;
}

int32_t lbm_next_step_odd(const lbm_ctx* c) { return c ? c->odd : -1; }

lbm_status lbm_column_max(lbm_ctx* c, float* m) {
    const Range range("lbm_column_max");
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (!m) return arg_fail(c, "m is NULL");
    cudaError_t e = launch_column_max(c->kp, kind(&c->p), c->odd != 0, c->v, m, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "column_max launch");
    return LBM_OK;
}

lbm_status lbm_front_of_columns(const float* m, int32_t nx, double threshold, int32_t x0,
                                int32_t H, int32_t periodic_x, double* out2, void* stream) {
    if (!m || !out2) return arg_fail(nullptr, "m and out2 must not be NULL");
    if (nx < 1 || H < 1 || x0 < 0 || x0 > nx || !isfinite(threshold))
        return arg_fail(nullptr, "nx >= 1, H >= 1, 0 <= x0 <= nx, finite threshold");
    cudaError_t e = launch_front_of_columns(
        m, nx, threshold, x0, (double)H, front_xlim(nx, x0, periodic_x ? LBM_FLAG_PERIODIC_X : 0),
        out2, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        snprintf(g_err, sizeof g_err, "front_of_columns launch: %s", cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

int64_t lbm_get_step(const lbm_ctx* c) { return c ? c->step : -1; }

lbm_status lbm_sync(lbm_ctx* c) {
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sync");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "sync");
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) { free(c); }

int32_t lbm_debug_build(void) {
#ifdef LBM_DEBUG
    return 1;
#else
    return 0;
#endif
}

lbm_status lbm_debug_record(lbm_ctx* c, int64_t out[4]) {
    if (!c) return arg_fail(nullptr, "ctx is NULL");
    if (!out) return arg_fail(c, "out is NULL");
    DbgRecord r;
    cudaError_t e = cudaMemcpyAsync(&r, dbg_record(c->v.devflags), sizeof r,
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "debug record copy");
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "debug record sync");
    if (r.count == 0) r = DbgRecord{};
    out[0] = (int64_t)r.count;
    out[1] = r.site;
    out[2] = r.off;
    out[3] = r.extent;
    return LBM_OK;
}

}  // extern "C"
