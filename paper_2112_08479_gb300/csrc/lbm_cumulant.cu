// lbm_cumulant.cu -- fused AA stream + collide kernel of the D3Q27 cumulant
// fluid (Sec. 2.3.1 "VirtualFluids", Eq. 52-58) with the D3Q7 scalar and the
// Boussinesq force.
//
// The collision (Eq. 54-58 with all rates of order >= 3 equal to 1, built
// from the Gaussian central moments of the relaxed covariance) is
// collide_cumulant in lbm_cumulant_collide.cuh.
#include <type_traits>

#include "lbm_cumulant_collide.cuh"
#include "lbm_internal.h"

namespace lbmgpu {

// Minimum resident blocks per SM for the register allocator: the D3Q27 FCM
// scalar holds more live values, so its instantiation gets its own setting;
// 3 (168 registers, 36-56 bytes of spills) measured 14.1 G node updates/s
// against 11.9 for 2 and 11.3 for 4 (128 registers, ~200 bytes of spills).
#ifndef LBM_Q27_MINB
#define LBM_Q27_MINB 3
#endif
#ifndef LBM_CUM_MINB
#define LBM_CUM_MINB LBM_STEP_MINB
#endif
#ifndef LBM_CUM_WSPLIT
#define LBM_CUM_WSPLIT 1
#endif

// With the D3Q27 scalar the factorized-central-moment collision needs, of
// the 27 pre-collision scalar populations, only chi, their first moments and
// (for the closing sum of the rest population) the populations themselves
// at the very end.  So the scalar is read, reduced to those four numbers and
// dropped; the fluid collides and is stored; then the scalar is read again
// (the same elements, which no other thread writes within the step) and
// collided: 27 values fewer live across the fluid collision.  Same arithmetic
// as collide_cumulant<27>.
template <bool ODD, bool SAVE, typename S, bool W, typename Off>
__device__ __forceinline__ void cumulant_fcm_step_body(const KParams& kp, S* __restrict__ f,
                                                       S* __restrict__ phi,
                                                       float* __restrict__ save,
                                                       const Stencil& st) {
    const unsigned n = st.n;
    constexpr bool R32 = rest32<S, 27>();
    constexpr bool s16 = !std::is_same<S, float>::value;
    float chs = 0.0f, jpx, jpy, jpz;
    {
        float pv[27];
        gather<27, ODD, S, 0, R32, W, Off>(kp, phi, st, pv);
        if (SAVE) {
#pragma unroll
            for (int k = 0; k < 27; ++k)
                save_pop(kp, save, 54, 27 + k, n, s16 ? pv[k] * kp.isp : pv[k]);
        }
        if (s16) {
#pragma unroll
            for (int k = 0; k < 27; ++k) pv[k] *= kp.isp;
        }
#pragma unroll
        for (int k = 0; k < 27; ++k) chs += pv[k];
        scalar_first_moments27(pv, jpx, jpy, jpz);
    }
    float fv[27];
    gather<27, ODD, S, 0, false, W, Off>(kp, f, st, fv);
    if (SAVE) {
#pragma unroll
        for (int i = 0; i < 27; ++i) save_pop(kp, save, 54, i, n, s16 ? fv[i] * kp.isf : fv[i]);
    }
    const bool collide = !(kp.flags & LBM_FLAG_NO_COLLIDE);
    float chit = 0.0f, chi = 1.0f, hx = 0.0f, hy = 0.0f, hz = 0.0f;
    if (s16) {
#pragma unroll
        for (int i = 0; i < 27; ++i) fv[i] *= kp.isf;
    }
    if (collide) cumulant_fluid<false>(kp, fv, chs, chit, chi, hx, hy, hz);
    if (s16) {
#pragma unroll
        for (int i = 0; i < 27; ++i) fv[i] *= kp.sf;
    }
    scatter<27, ODD, S, 0, false, W, Off>(kp, f, st, fv);
    // keep the second read of the scalar after the fluid's collision (the
    // compiler would otherwise issue it early and hold its values live again)
    asm volatile("" ::: "memory");
    // (held in registers all at once: reading, relaxing and storing the
    // scalar in groups of opposite pairs spills nothing but measured 7-17 %
    // slower, the loads of each group waiting behind the stores of the last)
    float pv[27];
    gather<27, ODD, S, 0, R32, W, Off>(kp, phi, st, pv);
    if (s16) {
#pragma unroll
        for (int k = 0; k < 27; ++k) pv[k] *= kp.isp;
    }
    if (collide) collide_fcm27(kp, pv, chit, chi, hx, hy, hz, jpx, jpy, jpz);
    if (s16) {
#pragma unroll
        for (int k = 0; k < 27; ++k) pv[k] *= kp.sp;
    }
    if constexpr (R32) feed_rest<S>(pv);
    scatter<27, ODD, S, 0, R32, W, Off>(kp, phi, st, pv);
}

template <bool ODD, bool SAVE, typename S, int SL, bool W, typename Off>
__device__ __forceinline__ void cumulant_step_body(const KParams& kp, S* __restrict__ f,
                                                   S* __restrict__ phi, float* __restrict__ save,
                                                   const Stencil& st) {
    const unsigned n = st.n;
    constexpr int NS = ScalarLat<SL>::NS;
    constexpr bool R32 = rest32<S, SL>();
    float fv[27], pv[NS];
    gather<27, ODD, S, 0, false, W, Off>(kp, f, st, fv);
    gather<NS, ODD, S, 0, R32, W, Off>(kp, phi, st, pv);
    constexpr bool s16 = !std::is_same<S, float>::value;   // populations in storage units
    constexpr bool fold = s16 && SL == 7;                  // the collision applies the scales
    if (SAVE) {
#pragma unroll
        for (int i = 0; i < 27; ++i)
            save_pop(kp, save, 27 + NS, i, n, s16 ? fv[i] * kp.isf : fv[i]);
#pragma unroll
        for (int k = 0; k < NS; ++k)
            save_pop(kp, save, 27 + NS, 27 + k, n, s16 ? pv[k] * kp.isp : pv[k]);
    }
    if (s16 && !fold) {
#pragma unroll
        for (int i = 0; i < 27; ++i) fv[i] *= kp.isf;
#pragma unroll
        for (int k = 0; k < NS; ++k) pv[k] *= kp.isp;
    }
    if (!(kp.flags & LBM_FLAG_NO_COLLIDE)) collide_cumulant<SL, fold>(kp, fv, pv);
    if (s16 && !fold) {
#pragma unroll
        for (int i = 0; i < 27; ++i) fv[i] *= kp.sf;
#pragma unroll
        for (int k = 0; k < NS; ++k) pv[k] *= kp.sp;
    }
    if constexpr (R32) feed_rest<S>(pv);
    scatter<27, ODD, S, 0, false, W, Off>(kp, f, st, fv);
    scatter<NS, ODD, S, 0, R32, W, Off>(kp, phi, st, pv);
}

// One node per thread.  On odd steps the blocks with no wall neighbour
// (uniform per block) take a body without the wall selects (D3Q7 scalar:
// measured 0.6-0.9 % faster; with the D3Q27 scalar the second body costs
// registers and was 4 % slower, so that instantiation keeps one body).
template <bool ODD, bool SAVE, typename S, int SL, typename Off = unsigned>
__global__ void __launch_bounds__(128, SL == 27 ? LBM_Q27_MINB : LBM_CUM_MINB) cumulant_step_kernel(KParams kp, S* __restrict__ f,
                                                            S* __restrict__ phi,
                                                            float* __restrict__ save) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const Stencil st = make_stencil(kp, x, blockIdx.y, blockIdx.z);
    if constexpr (SL == 27) {
        cumulant_fcm_step_body<ODD, SAVE, S, true, Off>(kp, f, phi, save, st);
    } else {
        if (!ODD || (LBM_CUM_WSPLIT && block_interior(kp)))
            cumulant_step_body<ODD, SAVE, S, SL, false, Off>(kp, f, phi, save, st);
        else
            cumulant_step_body<ODD, SAVE, S, SL, true, Off>(kp, f, phi, save, st);
    }
}

template <typename S, int SL>
static cudaError_t launch_cumulant_typed(const KParams& kp, bool odd, S* f, S* phi, float* save,
                                        cudaStream_t st) {
    dim3 block(128), grid((kp.nx + 127) / 128, kp.ny, kp.nz);
    if (kp.wide) {   // (Q + NS) N >= 2^32: 64-bit element offsets; no saved steps
        if (save) return cudaErrorInvalidValue;
        if (odd) cumulant_step_kernel<true, false, S, SL, size_t><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
        else cumulant_step_kernel<false, false, S, SL, size_t><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
        return cudaGetLastError();
    }
    if (save) {
        if (odd) cumulant_step_kernel<true, true, S, SL><<<grid, block, 0, st>>>(kp, f, phi, save);
        else cumulant_step_kernel<false, true, S, SL><<<grid, block, 0, st>>>(kp, f, phi, save);
    } else {
        if (odd) cumulant_step_kernel<true, false, S, SL><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
        else cumulant_step_kernel<false, false, S, SL><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
    }
    return cudaGetLastError();
}

template <int SL>
static cudaError_t launch_cumulant_sl(const KParams& kp, int storage, bool odd, void* f, void* phi,
                                      float* save, cudaStream_t st) {
    switch (storage) {
        case LBM_FP32: return launch_cumulant_typed<float, SL>(kp, odd, (float*)f, (float*)phi, save, st);
        case LBM_FP16S:
            return launch_cumulant_typed<__half, SL>(kp, odd, (__half*)f, (__half*)phi, save, st);
        case LBM_BF16S:
            return launch_cumulant_typed<__nv_bfloat16, SL>(kp, odd, (__nv_bfloat16*)f,
                                                            (__nv_bfloat16*)phi, save, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cumulant_step(const KParams& kp, int storage, int scalar, bool odd, void* f,
                                 void* phi, float* save, cudaStream_t st) {
    if (scalar == LBM_SCALAR_Q7) return launch_cumulant_sl<7>(kp, storage, odd, f, phi, save, st);
    if (scalar == LBM_SCALAR_Q27) return launch_cumulant_sl<27>(kp, storage, odd, f, phi, save, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbmgpu
