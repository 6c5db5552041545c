// lbm_internal.h -- host-side launchers shared by the C-ABI layer and the
// kernel translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_common.cuh"

namespace lbmgpu {

// Device-side diagnostics record written by the finalize kernel.
struct DevDiag {
    double front, front_node, Fw, mass_delta, scalar_mass;
};

// Front of a canonical state and its derivative with respect to the
// column maxima it interpolates between (lbm_front_adjoint).
struct FrontGrad {
    double value;     // (x_f + 1/2 - x0) / H
    double g0, g1;    // d value / d m(x), d value / d m(x + 1)
    int x, z0, z1;    // crossing column x and the z of the maxima of x and x + 1
    int valid;        // 1 when x + 1 < nx (the interpolated case)
};

// Workspace views handed to the launchers.
struct Views {
    void* f;              // Q * N storage elements
    void* phi;            // 7 * N storage elements
    float* stage;         // N floats: staging of a caller scalar field
    float* chibar;        // nx * nz floats: span-averaged scalar
    unsigned* colmax;     // nx order-preserving keys of max_z chibar
    double* part;         // 2 doubles per diagnostics block
    float* fwpart;        // 2 floats per diagnostics block
    DevDiag* ddiag;       // one record
    FrontGrad* fgrad;     // one record
    int* devflags;        // sticky device flags
    unsigned diag_blocks; // number of diagnostics blocks
};

// Per-model step launchers (lbm_bgk.cu, lbm_cumulant.cu).
cudaError_t launch_bgk_step(const KParams& kp, int storage, int scalar, bool odd, void* f,
                            void* phi, float* save, cudaStream_t st);
cudaError_t launch_cumulant_step(const KParams& kp, int storage, int scalar, bool odd, void* f,
                                 void* phi, float* save, cudaStream_t st);

// Model, scalar lattice and storage select the kernel (the pairs the ABI
// accepts: BGK with D3Q7 or D3Q6, cumulant with D3Q7 or D3Q27).
struct Kind {
    int model, scalar, storage;
};

// The TMA-staged step kernels (lbm_staged.cu): whether they serve this box
// and kind, and their launcher.
bool staged_step_applies(const KParams& kp, Kind k);
cudaError_t launch_staged_step(const KParams& kp, Kind k, bool odd, void* f, void* phi,
                               cudaStream_t st);

// odd: parity of the AA step.
cudaError_t launch_step(const KParams& kp, Kind k, bool odd, void* f, void* phi, float* save,
                        cudaStream_t st);
cudaError_t launch_init(const KParams& kp, Kind k, const Views& v, const float* chi0, int x0,
                        double amp, uint64_t seed, cudaStream_t st);
cudaError_t launch_macros(const KParams& kp, Kind k, bool odd, const Views& v, float* rho,
                          float* u, float* chi, cudaStream_t st);
cudaError_t launch_get_state(const KParams& kp, Kind k, bool odd, const Views& v, float* dst,
                             cudaStream_t st);
cudaError_t launch_set_state(const KParams& kp, Kind k, const Views& v, const float* src,
                             cudaStream_t st);
cudaError_t launch_diag(const KParams& kp, Kind k, bool odd, const Views& v, double threshold,
                        int x0, double H, cudaStream_t st);
cudaError_t launch_fw_accumulate(const KParams& kp, Kind k, bool odd, const Views& v,
                                 double* acc, double weight, cudaStream_t st);
cudaError_t launch_adjoint_step(const KParams& kp, const float* state, const float* lam_next,
                                float* lam, double* dcs, float wfw, float dAdCs, cudaStream_t st);
cudaError_t launch_push_step(const KParams& kp, const float* src, float* dst, cudaStream_t st);
cudaError_t launch_cumulant_adjoint_step(const KParams& kp, const float* state,
                                         const float* lam_next, float* lam, float wfw,
                                         cudaStream_t st);
cudaError_t launch_cumulant_push_step(const KParams& kp, const float* src, float* dst,
                                      cudaStream_t st);
cudaError_t launch_front_adjoint(const KParams& kp, int Q, int NS, const Views& v,
                                 const float* state, float* lam, double* value, double threshold,
                                 int x0, double H, cudaStream_t st);
cudaError_t launch_adjoint_chi0(const KParams& kp, int Q, const float* lam0, float* grad,
                                cudaStream_t st);

unsigned diag_block_count(int nx, int nz);

// x-slabs (lbm_slab.cu, lbm_aux.cu): face buffers of the halo exchange and
// the column maxima of the front.
size_t halo_elems(int Q, int NS, int ny, int nz);
cudaError_t launch_halo(const KParams& kp, Kind k, int face, bool pack, void* f, void* phi,
                        void* buf, cudaStream_t st);
cudaError_t launch_column_max(const KParams& kp, Kind k, bool odd, const Views& v, float* m,
                              cudaStream_t st);
cudaError_t launch_front_of_columns(const float* m, int nx, double thr, int x0, double H,
                                    int xlim, double* out, cudaStream_t st);

}  // namespace lbmgpu
