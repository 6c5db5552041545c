/*
 * lbm.h -- C ABI of the GB300 lock-exchange lattice Boltzmann library.
 *
 * The library advances the coupled fluid / scalar lattice Boltzmann model of
 * Adekanye et al., "GPU accelerated LBM simulations of dilute gravity
 * currents" (arXiv 2112.08479), one fused stream + collide kernel per time
 * step, on one CUDA device:
 *
 *   fluid   D3Q19 BGK with a Smagorinsky eddy viscosity and Guo forcing
 *           (Sec. 2.3.1, Eq. 17-26, 32-34), or D3Q27 cumulant
 *           (Sec. 2.3.1 "VirtualFluids", Eq. 52-58);
 *   scalar  D3Q7 BGK advection-diffusion (Eq. 27-30, 35);
 *   force   Boussinesq body force F = g' chi e^g (Sec. 2.1, Eq. 11);
 *   walls   half-way bounce-back at both x ends and both z ends, periodic
 *           in y (Sec. 2.5).
 *
 * Conventions shared by every entry point:
 *  - Lattice units, dx = dt = 1.  Node index n = x + nx * (y + ny * z).
 *  - Ownership: the caller allocates every device buffer, including the
 *    workspace handed to lbm_init; the library allocates no device memory.
 *    lbm_ctx is a small host object owned by the library.
 *  - Execution: all device work is enqueued on the CUDA stream given to
 *    lbm_init and is asynchronous, except where an entry point says it
 *    synchronises.  Device pointers must be usable on that stream's device.
 *  - Errors: arguments are checked on the host before anything is enqueued
 *    (LBM_ERR_ARG, nothing happens).  Launch failures return LBM_ERR_CUDA.
 *    Asynchronous faults and the device-side sticky flags (non-finite value,
 *    rho <= 0) are reported by the next synchronising call (lbm_diag,
 *    lbm_sync).  Nothing aborts, exits or traps.
 *  - Canonical state layout (lbm_get_state / lbm_set_state / adjoint):
 *    FP32, direction-major, [Q + NS][N]: rows 0..Q-1 hold f_i - w_i of the
 *    pre-collision (streamed) fluid populations, rows Q..Q+NS-1 hold
 *    Phi_k - w_k of the NS scalar populations (w the lattice weights; both
 *    sets are held as deviations from their rest state rho = 1, chi = 1).
 *    Direction orders: D3Q19 as in Eq. 23; D3Q27 as Eq. 23 followed by the
 *    corners (1,1,1), (-1,-1,-1), (1,1,-1), (-1,-1,1), (1,-1,1), (-1,1,-1),
 *    (-1,1,1), (1,-1,-1); D3Q7 rest, +x, -x, +y, -y, +z, -z; D3Q6 as D3Q7
 *    without the rest population (Eq. 31).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbm_status {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,       /* invalid argument; nothing was enqueued */
    LBM_ERR_CUDA = 2,      /* a CUDA call or launch failed */
    LBM_ERR_NOMEM = 3,     /* workspace smaller than lbm_workspace_bytes */
    LBM_ERR_UNSTABLE = 4,  /* sticky device flag: non-finite value or rho <= 0 */
    LBM_ERR_STATE = 5,     /* call not valid in the context's current state */
    LBM_ERR_TIMEOUT = 6,   /* a bounded wait gave up */
    LBM_ERR_BOUNDS = 7     /* debug build only: an index check failed (lbm_debug_record) */
} lbm_status;

typedef enum lbm_model {
    LBM_BGK_SMAG_Q19 = 0,  /* Sec. 2.3.1 RAFSINE physics: Eq. 21-26, 32-34 */
    LBM_CUMULANT_Q27 = 1   /* Sec. 2.3.1 VirtualFluids physics: Eq. 54-58, all
                              rates of order >= 3 equal to 1 */
} lbm_model;

typedef enum lbm_scalar {
    LBM_SCALAR_Q7 = 0,   /* D3Q7 BGK, c_sPhi^2 = 1/4 (both models) */
    LBM_SCALAR_Q6 = 1,   /* D3Q6 BGK as printed in Eq. 29-31 (RAFSINE): w = 1/6,
                            c_s^2 = 1/3, no rest population; BGK model only */
    LBM_SCALAR_Q27 = 2   /* D3Q27 factorized central moments (Eq. 37-51,
                            VirtualFluids), all rates of order >= 2 equal to 1;
                            cumulant model only */
} lbm_scalar;

typedef enum lbm_storage {
    LBM_FP32 = 0,   /* populations stored as FP32: f - w and Phi - w */
    LBM_FP16S = 1,  /* FP16, scale_f * (f - w) and scale_phi * (Phi - LBM_SCALAR_CHI16 w)
                       (= Phi - w), RN rounding */
    LBM_BF16S = 2   /* BF16, same shifts and scales, RN rounding */
} lbm_storage;

/* 16-bit storage holds the scalar populations as deviations from the field
   chi = LBM_SCALAR_CHI16: 1, the heavy fluid, so Phi - w as in FP32.  (A
   build constant of the storage format: 1/2, the middle of chi's range,
   halves the largest stored magnitude but measured no smaller FP16 front
   error on average over three lock-exchange boxes.)  The FP32 forms (FP32
   storage, lbm_get_state / lbm_set_state, saved steps) are Phi - w. */
#define LBM_SCALAR_CHI16 1.0

/* lbm_params.flags */
#define LBM_FLAG_NO_COLLIDE 1  /* skip every collision: pure streaming (tests) */
#define LBM_FLAG_PERIODIC_X 2  /* periodic instead of walls at the x ends */
#define LBM_FLAG_PERIODIC_Z 4  /* periodic instead of walls at the z ends */
#define LBM_FLAG_ONE_NODE 8    /* one node per thread in the step kernels (test hook: the
                                  two- and four-node kernels are checked against it) */
#define LBM_FLAG_TMA_STAGED 16 /* cumulant model, D3Q7 scalar, 16-bit storage, nx a multiple
                                  of 256: run each step through the TMA-staged kernel (row
                                  segments moved by bulk copies through shared memory by a
                                  producer warp); same results bit for bit, measured slower
                                  than the default kernel on GB300; ignored elsewhere */
#define LBM_FLAG_TEST_STALL 32 /* test hook of the failure path of LBM_FLAG_TMA_STAGED: each
                                  block's first tile is announced on its barrier but never
                                  copied, so its wait cannot end; every wait gives up after
                                  0.1 s, the kernel sets LBM_DEVFLAG_TIMEOUT and returns
                                  (lbm_diag then reports LBM_ERR_TIMEOUT); no fault, no hang */
#define LBM_FLAG_TEST_BOUNDS 64 /* test hook of the index checks of the debug build (rejected
                                   with LBM_ERR_ARG by the release build): every check uses
                                   half of its array's true extent, so the in-bounds accesses
                                   to the upper half of each array fail the check, are
                                   recorded and skipped; no access leaves its array */

/* sticky device flags reported in lbm_diagnostics.flags */
#define LBM_DEVFLAG_NONFINITE 1   /* a macroscopic value was NaN or Inf */
#define LBM_DEVFLAG_RHO_NONPOS 2  /* rho <= 0 at some node */
#define LBM_DEVFLAG_TIMEOUT 4     /* a step kernel could not move its populations
                                     through shared memory (a bounded wait for its
                                     own bulk copies gave up, or the shared memory
                                     was misaligned): the step is incomplete */
#define LBM_DEVFLAG_BOUNDS 8      /* debug build: an index check failed and its access
                                     was skipped (lbm_debug_record) */

typedef struct lbm_params {
    int32_t nx, ny, nz;       /* nodes; 1 <= nx, ny, nz; nx*ny*nz < 2^31; ny, nz <= 65535.
                                 Boxes with (Q+NS)*nx*ny*nz >= 2^32 step with 64-bit
                                 element offsets; lbm_step_save and the adjoint entry
                                 points need (Q+NS)*nx*ny*nz < 2^32 (LBM_ERR_STATE) */
    int32_t model;            /* lbm_model */
    int32_t storage;          /* lbm_storage */
    int32_t flags;            /* LBM_FLAG_* */
    double nu;                /* molecular viscosity, tau0 = 3 nu + 1/2 (Eq. 25); > 0 */
    double D;                 /* molecular diffusivity, tau_Phi = 1/2 + 4 D (Eq. 30
                                 with c_sPhi^2 = 1/4 on D3Q7); > 0 */
    double cs_smag;           /* classical Smagorinsky constant, nu_T = (C_s)^2 |S|
                                 (Eq. 32, Delta = 1); BGK only; >= 0 */
    double sc_t;              /* turbulent Schmidt number, D_eff = D + nu_T / Sc_T
                                 (Eq. 35); > 0 */
    double gprime;            /* reduced gravity g' in F = g' chi e^g (Eq. 11) */
    double eg[3];             /* gravity direction e^g, (0, 0, -1) in the paper */
    double omega_bulk;        /* cumulant: relaxation rate of the second-order trace
                                 (1 = equilibrium each step); (0, 2) */
    int32_t x0;               /* lock gate: chi0 = 1 for x < x0 (Table 1); 0..nx */
    int32_t H;                /* depth used to scale the front, > 0 (usually nz) */
    double noise_amp;         /* chi0 += noise_amp * U(-1, 1) on column x0 - 1 */
    uint64_t seed;            /* noise draw for node n: splitmix64(seed ^ n) */
    double front_threshold;   /* span-averaged chi threshold of the front (0.02) */
    double scale_f;           /* 16-bit storage scale of f - w (power of two) */
    double scale_phi;         /* 16-bit storage scale of Phi - w (power of two) */
    int32_t scalar;           /* lbm_scalar */
    int32_t x_offset;         /* x-slab of a larger box: global x of local column 0
                                 (0 for a whole box) */
    int32_t nx_global;        /* x-slab: nx of the whole box (0: nx, a whole box).  With
                                 nx_global > nx the local x ends are slab faces: walls
                                 to the kernels, made fluid by the halo exchange of
                                 lbm_halo_pack / lbm_halo_unpack around every odd step;
                                 x0, the lock noise (keyed by the global node index)
                                 and the front refer to the whole box */
    int32_t pad_;
} lbm_params;

typedef struct lbm_diagnostics {
    double front;        /* (x_f + 1/2 - x0) / H, Sec. 3.1 (an x-slab: over its own
                            columns, in box coordinates; the box's front comes
                            from lbm_column_max of every slab) */
    double front_node;   /* x_f in node coordinates, -1 when no column reaches
                            the threshold; searched over all x with walls at
                            the x ends, over x < (nx + x0) / 2 with
                            LBM_FLAG_PERIODIC_X (the half of the ring ahead of
                            the lock) */
    double Fw;           /* bottom-wall friction sum_{x,y} tau_w, Eq. 62-64,
                            lattice units, streamwise component */
    double mass_delta;   /* sum over nodes of rho - 1 (FP64 reduction) */
    double scalar_mass;  /* sum over nodes of chi (FP64 reduction) */
    int64_t step;        /* time step the values belong to */
    int32_t flags;       /* LBM_DEVFLAG_* seen since lbm_init (sticky) */
    int32_t pad_;
} lbm_diagnostics;

typedef struct lbm_ctx lbm_ctx;

/* Human-readable name of a status code.  Never NULL. */
LBM_API const char* lbm_status_string(lbm_status s);

/* Last error message recorded on ctx (empty string when none). */
LBM_API const char* lbm_last_error(const lbm_ctx* ctx);

/* Checks p without touching the device.  LBM_OK or LBM_ERR_ARG. */
LBM_API lbm_status lbm_validate(const lbm_params* p);

/* Bytes of device workspace lbm_init needs for p; 0 when p is invalid.
 * The workspace holds what the flowchart of Sec. 2.3 (Fig. 3) exports to the
 * GPU once the set-up on the CPU is done: the distributions of the fluid and
 * the scalar (Eq. 17, 28), one copy each in the AA pattern, (Q + NS) * N *
 * (4 or 2) bytes; plus a few N- and nx-sized staging and reduction buffers
 * of the diagnostics (Sec. 3.1, 3.2). */
LBM_API size_t lbm_workspace_bytes(const lbm_params* p);

/* Creates a context over a caller-owned device workspace of `bytes` bytes
 * (>= lbm_workspace_bytes(p), 256-byte aligned) and enqueues the initial
 * condition of Sec. 2.5 on `cuda_stream` (a cudaStream_t, NULL = legacy
 * default stream): f = w (rho = 1, u = 0), chi0 = 1 for x < x0 else 0, plus
 * the noise on column x0 - 1, Phi_k = w_k chi0.  The workspace must outlive
 * the context.  *out is set only on LBM_OK. */
LBM_API lbm_status lbm_init(const lbm_params* p, void* workspace, size_t bytes,
                    void* cuda_stream, lbm_ctx** out);

/* Re-initialises the state from a caller-given scalar field chi0 (N floats,
 * host or device memory; copied on the stream before return of control to
 * the device queue): the fluid at rest, f = w (rho = 1, u = 0), and the
 * scalar at its equilibrium for that field, Phi_k = w_k chi0 (Eq. 29 at
 * u = 0), as in the initial condition of Sec. 2.5 with chi0 in place of the
 * lock field.  Resets the step counter. */
LBM_API lbm_status lbm_set_scalar(lbm_ctx* ctx, const float* chi0);

/* Advances nsteps >= 0 time steps (Eq. 17): one fused in-place kernel per
 * step (AA pattern: even steps collide in place, odd steps gather from and
 * scatter to the neighbours).  Asynchronous. */
LBM_API lbm_status lbm_step(lbm_ctx* ctx, int32_t nsteps);

/* One time step that also writes the pre-collision state of the current
 * step, in the canonical layout, to state_out ((Q + NS) * N floats, device).
 * Used to record the forward trajectory for the adjoint. */
LBM_API lbm_status lbm_step_save(lbm_ctx* ctx, float* state_out);

/* Macroscopic fields of the current state (Eq. 19, 20 with the half-force
 * shift, 27): rho (N floats), u (3 * N floats, component-major [3][N]), chi
 * (N floats).  Device buffers; any may be NULL.  Asynchronous. */
LBM_API lbm_status lbm_macros(lbm_ctx* ctx, float* rho, float* u, float* chi);

/* Diagnostics of the current state (Sec. 3.1 front, Eq. 62-64 F_w, FP64
 * mass and scalar budgets) into a host struct.  Synchronises the stream.
 * Returns LBM_ERR_TIMEOUT when LBM_DEVFLAG_TIMEOUT is set, otherwise
 * LBM_ERR_UNSTABLE when another sticky device flag is set (the struct is
 * still filled in both cases), LBM_ERR_CUDA on an asynchronous fault. */
LBM_API lbm_status lbm_diag(lbm_ctx* ctx, lbm_diagnostics* out_host);

/* Adds weight * F_w(current state) to *acc_dev (one device double).
 * Asynchronous.  Used for the time-integrated friction objective. */
LBM_API lbm_status lbm_fw_accumulate(lbm_ctx* ctx, double* acc_dev, double weight);

/* Copies the current state to dst ((Q + NS) * N floats, canonical layout,
 * device): the streamed, pre-collision distributions f_i(x, t) and Phi_k(x, t)
 * of Eq. 17 and 28 at the current step, i.e. the data the flowchart of
 * Sec. 2.3 (Fig. 3) transfers back from the GPU for output.  Asynchronous. */
LBM_API lbm_status lbm_get_state(lbm_ctx* ctx, float* dst);

/* Loads a state in the canonical layout (device): pre-collision
 * distributions of Eq. 17 and 28 as lbm_get_state writes them (the export
 * to the GPU of Fig. 3, from a caller's state instead of the initial
 * condition of Sec. 2.5), and sets the step counter.  Asynchronous. */
LBM_API lbm_status lbm_set_state(lbm_ctx* ctx, const float* src, int64_t step);

/* One reverse step of the discrete adjoint of the time step with the D3Q7
 * scalar and the Boussinesq force, for either fluid (BGK-Smagorinsky,
 * Eq. 17-35; cumulant, Eq. 54-58 and 28-30), in FP32 arithmetic:
 *   lam_n = (dT/ds_n)^T lam_next + w_fw * dF_w(s_n)/ds_n,
 *   *dJdCs_dev += lam_next . dT/dC_s (s_n)   (BGK; the cumulant model has
 *                                            no C_s and adds nothing),
 * where T is the time step of lbm_step, s_n = state_n (canonical layout,
 * device, (Q + NS) * N floats) is the state it was applied to, and lam_next,
 * lam_n are adjoint states in the canonical layout (device, (Q + NS) * N
 * floats; lam_next == NULL means zero).  lam_n must not alias lam_next or
 * state_n.  dJdCs_dev: one device double, accumulated.  Asynchronous.
 * LBM_ERR_STATE for the D3Q6 and D3Q27 scalars. */
LBM_API lbm_status lbm_adjoint_step(lbm_ctx* ctx, const float* state_n, const float* lam_next,
                            float* lam_n, double* dJdCs_dev, double w_fw);

/* Forward pass of the time-integrated bottom friction J = sum_n F_w(s_n):
 * advances nsteps >= 0 steps from the current state s_0, adding F_w of each
 * new state to *J_dev (one device double; NULL skips the sum, for objectives
 * of the final state only), and, when ckpt is not NULL, copies the state
 * before relative step n to ckpt + (n / K) (Q + NS) N for every n % K == 0
 * (canonical layout, device; ceil(nsteps / K) states).  Asynchronous. */
LBM_API lbm_status lbm_objective_forward(lbm_ctx* ctx, int32_t nsteps, int32_t K, float* ckpt,
                                         double* J_dev);

/* One reverse segment of the adjoint of J (either fluid with the D3Q7
 * scalar, FP32 storage):
 * from the checkpoint ckpt = s_{n0}, recomputes s_{n0+1} .. s_{n0+k-1} into
 * seg + j (Q + NS) N (j = 1 .. k-1; seg holds k states, slot 0 unused) with
 * an out-of-place step of the same arithmetic, then applies k adjoint steps
 * backwards: on entry lam holds lam_{n0+k}, on return lam_{n0}; the
 * friction of every state s_n with n >= 1 enters with weight w_fw (1 for the
 * time-integrated friction, 0 for an objective of the final state, e.g. the
 * front of lbm_front_adjoint).  tmp: a second adjoint buffer, distinct from
 * lam.  *dJdCs_dev accumulates the C_s derivative.  Asynchronous.
 * LBM_ERR_STATE for 16-bit storage or the D3Q6 and D3Q27 scalars. */
LBM_API lbm_status lbm_adjoint_segment(lbm_ctx* ctx, const float* ckpt, int64_t n0, int32_t k,
                                       float* seg, float* lam, float* tmp, double* dJdCs_dev,
                                       double w_fw);

/* The two halves of lbm_adjoint_segment, for callers that overlap the
 * recompute of one segment with the adjoint sweep of the next (two streams):
 *
 * lbm_recompute_segment: from ckpt = s_{n0}, writes s_{n0+1} .. s_{n0+k-1}
 * into seg + j (Q + NS) N, j = 1 .. k-1 (out-of-place steps of the same
 * arithmetic as lbm_step).
 *
 * lbm_adjoint_sweep: applies k adjoint steps backwards through ckpt (j = 0)
 * and seg + j (Q + NS) N (j = 1 .. k-1): on entry lam holds lam_{n0+k}, on
 * return lam_{n0}; w_fw, tmp and dJdCs_dev as for lbm_adjoint_segment.
 *
 * Both read ckpt and seg, both enqueue on `stream` (a cudaStream_t of the
 * context's device; NULL selects the context's stream) and neither
 * synchronises: ordering between the two calls (seg written before it is
 * swept, not overwritten while it is swept) is the caller's.  Device
 * buffers; LBM_ERR_STATE for 16-bit storage or the D3Q6 and D3Q27 scalars. */
LBM_API lbm_status lbm_recompute_segment(lbm_ctx* ctx, const float* ckpt, int32_t k, float* seg,
                                         void* stream);
LBM_API lbm_status lbm_adjoint_sweep(lbm_ctx* ctx, const float* ckpt, const float* seg,
                                     int64_t n0, int32_t k, float* lam, float* tmp,
                                     double* dJdCs_dev, double w_fw, void* stream);

/* Front position of a state and its derivative (Sec. 3.1 with reading R11:
 * chibar(x, z) = mean over y of chi, m(x) = max over z of chibar, x_f = the
 * largest searched x (see lbm_diagnostics.front_node) with m(x) >=
 * front_threshold, moved to the linear threshold crossing between x_f and
 * x_f + 1; value (x_f + 1/2 - x0) / H).  The
 * interpolated front is a continuous, piecewise smooth function of the
 * state, the smooth surrogate of the node-wise front used as an objective.
 * state: canonical layout ((Q + NS) * N floats, device).  front_dev: one
 * device double receiving the value, or NULL.  lam: NULL, or (Q + NS) * N
 * floats (device) receiving d value / d state: zero except on the scalar
 * rows of the 2 ny nodes (x_f, y, z0) and (x_f + 1, y, z1), z0 and z1 the
 * first z attaining m; zero everywhere when no column reaches the threshold
 * or x_f is the last searched column.  Any model, scalar lattice and storage.
 * Asynchronous. */
LBM_API lbm_status lbm_front_adjoint(lbm_ctx* ctx, const float* state, float* lam,
                                     double* front_dev);

/* Gradient with respect to the initial scalar field of a quantity whose
 * adjoint at step 0 is lam0: grad_chi0[n] = sum_k w_k lam0_Phi_k[n]
 * (since Phi_k = w_k chi0 at t = 0).  Device buffers.  Asynchronous. */
LBM_API lbm_status lbm_adjoint_chi0(lbm_ctx* ctx, const float* lam0, float* grad_chi0);

/* Diagnostics (as lbm_diag) of a state the caller holds in the canonical
 * layout (state: (Q + NS) * N floats, device), for callers that cannot
 * allocate device memory (an allocator callback or out-of-memory handler, a
 * pool fixed before this library loads): it needs no context and no
 * workspace and calls no cudaMalloc, cudaFree or allocating routine.  The
 * paper has no counterpart; this is a service of the library.
 * Its scratch is one fixed device array of 852,224 bytes inside the library,
 * present on every device that uses the library until it is unloaded; it
 * serves nx <= 16384 and ceil(nx / 128) * nz <= 32768 and returns
 * LBM_ERR_ARG beyond that (message in lbm_last_error(NULL)).  The first call
 * on each device looks up the array's device address; make that first call
 * with the device current.  Every call synchronises cuda_stream, so no call
 * may be made while that stream is being captured into a CUDA graph: such a
 * call returns LBM_ERR_ARG without enqueueing anything.  state must be
 * device memory of the current device (checked: LBM_ERR_ARG otherwise).
 * All calls share the array: calls that overlap on the GPU race and must be
 * serialised.  Enqueued on cuda_stream (its device must be current), then
 * synchronised; flags holds only what this call saw; LBM_ERR_UNSTABLE as
 * lbm_diag. */
LBM_API lbm_status lbm_diag_static(const lbm_params* p, const float* state, int64_t step,
                                   void* cuda_stream, lbm_diagnostics* out_host);

/* --- x-slab decomposition (one slab of a box per GPU) ---------------------
 * A box of nx_global columns is cut along x into slabs (lbm_params.x_offset,
 * nx_global); each slab is a context of its own, with walls at its x ends
 * to the step kernels.  After every step each pair of touching faces swaps
 * face buffers: both sides lbm_halo_pack their face, exchange the buffers,
 * then lbm_halo_unpack the neighbour's buffer into their face.  With
 * periodic x the last slab's face 1 touches the first slab's face 0.
 * Unpacking sets, at every face node (y, z), each population i whose c_ix
 * points into the slab to the neighbour's population opp(i) at its face node
 * (y - c_iy, z - c_iz) (y periodic; skipped where z - c_iz lies beyond the
 * top or bottom wall).  In the AA pattern a node at a face reads, for the
 * populations whose upwind node lies across the face, the slot a wall would
 * reflect (its own slot i), and pushes the populations leaving across the
 * face into the slots a wall would (its own slot opp(i)); the swap after an
 * even step puts the neighbour's post-collision populations where the next
 * odd step and any read of the state take them, the swap after an odd step
 * hands each side the populations the other pushed across (the streaming of
 * Eq. 17 across the face).  Steps, packs and unpacks of a slab execute in
 * stream order; results equal those of the whole box bit for bit.
 *
 * lbm_halo_bytes: bytes of one face buffer (device memory, caller-owned):
 * the populations with c_x = +1 of both lattices (5 + 1 for D3Q19 + D3Q7,
 * 9 + 1 cumulant + D3Q7, 9 + 9 cumulant + D3Q27), ny nz storage elements
 * each; 0 when p is invalid.
 * lbm_halo_pack: face 0 (x = 0) or 1 (x = nx - 1) of the current state into
 * buf.  lbm_halo_unpack: the buffer the neighbour packed from its touching
 * face, into face `face`.  Asynchronous.
 * lbm_next_step_odd: 1 when the context's next step is an odd AA step, 0
 * otherwise, -1 for NULL. */
LBM_API size_t lbm_halo_bytes(const lbm_params* p);
LBM_API lbm_status lbm_halo_pack(lbm_ctx* ctx, int32_t face, void* buf);
LBM_API lbm_status lbm_halo_unpack(lbm_ctx* ctx, int32_t face, const void* buf);
LBM_API int32_t lbm_next_step_odd(const lbm_ctx* ctx);

/* Column maxima of the front search (Sec. 3.1, reading R11) of the current
 * state: m[x] = max over z of the span-averaged chi of column x, for the
 * context's nx columns (device, nx floats).  A slab's columns, gathered in
 * x order over all slabs, give the whole box's.  Asynchronous. */
LBM_API lbm_status lbm_column_max(lbm_ctx* ctx, float* m);

/* Front of a whole box from its column maxima m[0 .. nx) (device):
 * out2[0] = (x_f + 1/2 - x0) / H and out2[1] = x_f as in lbm_diagnostics
 * (search window of periodic_x as there), two device doubles.  Enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default stream).  Asynchronous;
 * LBM_ERR_ARG (message in lbm_last_error(NULL)) for invalid arguments. */
LBM_API lbm_status lbm_front_of_columns(const float* m, int32_t nx, double threshold,
                                        int32_t x0, int32_t H, int32_t periodic_x,
                                        double* out2, void* stream);

/* Current step counter. */
LBM_API int64_t lbm_get_step(const lbm_ctx* ctx);

/* Synchronises the stream; reports asynchronous CUDA faults. */
LBM_API lbm_status lbm_sync(lbm_ctx* ctx);

/* Frees the host context (not the caller's workspace).  NULL is a no-op. */
LBM_API void lbm_destroy(lbm_ctx* ctx);

/* ---- index checks of the debug build -----------------------------------
 * The debug build of this library (liblbm_debug.so, compiled with
 * LBM_DEBUG) checks, before every population access of the step, halo,
 * adjoint and state-transfer kernels, that the accessed elements lie inside
 * their array (a population array of rows x N elements, the FP32 rest row,
 * a halo buffer, an adjoint or state buffer).  A failed check counts
 * itself, records the first failure, sets LBM_DEVFLAG_BOUNDS and skips the
 * access (a skipped load gives 0): an indexing error becomes a status the
 * host reads, never a memory fault.  lbm_diag returns LBM_ERR_BOUNDS once
 * the flag is set.  The release build compiles the checks to nothing.
 *
 * lbm_debug_build: 1 in the debug build, 0 in the release build.
 * lbm_debug_record: the context's record, out[0] = failed checks, out[1] =
 * site of the first failure (LBM_SITE_*), out[2] = its element offset in
 * its array, out[3] = the extent (elements) it was checked against; all 0
 * when no check failed, and always in the release build.  Synchronises the
 * context's stream; the workspace must still be allocated.  LBM_ERR_ARG for
 * NULL arguments.  (lbm_diag_static reads its state without these checks.) */
#define LBM_SITE_GATHER 1      /* one-node gather (step, diagnostics, state export) */
#define LBM_SITE_SCATTER 2     /* one-node scatter */
#define LBM_SITE_PAIR_LOAD 3   /* two-node gather */
#define LBM_SITE_PAIR_STORE 4  /* two-node scatter */
#define LBM_SITE_QUAD 5        /* four-node even step of 16-bit storage */
#define LBM_SITE_STAGED 6      /* TMA-staged step: bulk copies and direct accesses */
#define LBM_SITE_HALO 7        /* halo pack / unpack (state and face buffer) */
#define LBM_SITE_ADJOINT 8     /* adjoint kernels: saved states and adjoint fields */
#define LBM_SITE_STATE 9       /* initial condition, state import, saved steps */
LBM_API int32_t lbm_debug_build(void);
LBM_API lbm_status lbm_debug_record(lbm_ctx* ctx, int64_t out[4]);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
