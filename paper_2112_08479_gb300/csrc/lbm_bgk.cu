// lbm_bgk.cu -- fused AA stream + collide kernels of the D3Q19 BGK-Smagorinsky
// fluid with the D3Q7 scalar and the Boussinesq force.
//
// Per node and step (lattice units, c_s^2 = 1/3, populations held as
// deviations f - w from the rest weights so FP32 keeps its digits):
//   chi = sum_k Phi_k                                        (Eq. 27)
//   F = g' chi e^g                                           (Eq. 11)
//   rho = 1 + sum_i (f_i - w_i), rho u = sum_i c_i f_i + F/2  (Eq. 19-20, 52-53)
//   Pi = sum_i c_i c_i (f_i - feq_i) = M - (delta rho / 3) I - rho u u
//   q = |Pi|, tau = (tau0 + sqrt(tau0^2 + 18 sqrt2 C_s^2 q / rho)) / 2
//                                                   (Eq. 32-34, reading R3)
//   f*_i = f_i - (f_i - feq_i)/tau + (1 - 1/2tau) w_i [3 (c_i - u) + 9 (c_i.u) c_i].F
//                                                   (Eq. 17, 21, 22, 26)
//   tau_Phi = 1/2 + 4 (D + nu_T / Sc_T), nu_T = (tau - tau0) / 3   (Eq. 30, 35)
//   Phi*_k = Phi_k - (Phi_k - w_k chi (1 + 4 c_k.u)) / tau_Phi     (Eq. 28-29)
// followed by streaming (Eq. 17) in the AA pattern of lbm_common.cuh.
//
// The kernels are HBM-bound (about 2 flop per byte).  With nx even, one
// thread owns two x-adjacent nodes and moves every population row as aligned
// pairs (lbm_aa2.cuh): a warp reads and writes 256-byte row segments in FP32.
// With nx odd, one thread per node.  No shared memory, no tensor cores.
#include <type_traits>

#include "lbm_aa2.cuh"
#include "lbm_bgk_collide.cuh"
#include "lbm_internal.h"
#include "lbm_quad.cuh"

namespace lbmgpu {

template <bool ODD, bool SAVE, typename S, int SL, typename Off = unsigned>
__global__ void __launch_bounds__(128, LBM_STEP_MINB) bgk_step_kernel(KParams kp, S* __restrict__ f,
                                                       S* __restrict__ phi,
                                                       float* __restrict__ save) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const Stencil st = make_stencil(kp, x, blockIdx.y, blockIdx.z);
    const unsigned n = st.n;

    constexpr int NS = ScalarLat<SL>::NS, D0 = ScalarLat<SL>::D0;
    constexpr bool R32 = rest32<S, SL>();
    float fv[19], pv[NS];
    gather<19, ODD, S, 0, false, true, Off>(kp, f, st, fv);
    gather<NS, ODD, S, D0, R32, true, Off>(kp, phi, st, pv);
    constexpr bool s16 = !std::is_same<S, float>::value;   // populations in storage units
    if (SAVE) {
#pragma unroll
        for (int i = 0; i < 19; ++i) save_pop(kp, save, 19 + NS, i, n, s16 ? fv[i] * kp.isf : fv[i]);
#pragma unroll
        for (int k = 0; k < NS; ++k)
            save_pop(kp, save, 19 + NS, 19 + k, n,
                     s16 ? phi_canonical(kp, pv[k], ScalarLat<SL>::w(k)) : pv[k]);
    }
    if (!(kp.flags & LBM_FLAG_NO_COLLIDE)) collide_bgk<s16, SL>(kp, fv, pv);
    if constexpr (R32) feed_rest<S>(pv);
    scatter<19, ODD, S, 0, false, true, Off>(kp, f, st, fv);
    scatter<NS, ODD, S, D0, R32, true, Off>(kp, phi, st, pv);
}


#ifndef LBM_BGK_ZSPLIT
#define LBM_BGK_ZSPLIT 1
#endif
#ifndef LBM_BGK_FAST
#define LBM_BGK_FAST 1
#endif

// The 16-bit instantiations are issue-bound rather than HBM-bound, so they
// may trade registers for resident warps differently (LBM_STEP2_MINB16).
#ifndef LBM_STEP2_MINB16
#define LBM_STEP2_MINB16 LBM_STEP2_MINB
#endif

template <bool ODD, bool SAVE, typename S, int SL, bool ZW, bool FAST, typename Off>
__device__ __forceinline__ void bgk_step2_body(const KParams& kp, S* __restrict__ f,
                                               S* __restrict__ phi, float* __restrict__ save,
                                               const Stencil2& st) {
    constexpr int NS = ScalarLat<SL>::NS, D0 = ScalarLat<SL>::D0;
    constexpr bool R32 = rest32<S, SL>();
    float f0[19], f1[19], p0[NS], p1[NS];
    gather2<19, ODD, S, 0, false, ZW, FAST, Off>(kp, f, st, f0, f1);
    gather2<NS, ODD, S, D0, R32, ZW, FAST, Off>(kp, phi, st, p0, p1);
    constexpr bool s16 = !std::is_same<S, float>::value;   // populations in storage units
    if (SAVE && st.active) {
        const unsigned N = kp.N;
        const float a = s16 ? kp.isf : 1.0f;
#pragma unroll
        for (int i = 0; i < 19; ++i)
            *reinterpret_cast<float2*>(save + (size_t)i * N + st.n) = make_float2(a * f0[i], a * f1[i]);
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const float w = ScalarLat<SL>::w(k);
            *reinterpret_cast<float2*>(save + (size_t)(19 + k) * N + st.n) =
                s16 ? make_float2(phi_canonical(kp, p0[k], w), phi_canonical(kp, p1[k], w))
                    : make_float2(p0[k], p1[k]);
        }
    }
    if (!(kp.flags & LBM_FLAG_NO_COLLIDE)) {
        collide_bgk<s16, SL>(kp, f0, p0);
        collide_bgk<s16, SL>(kp, f1, p1);
    }
    if constexpr (R32) feed_rest2<S>(p0, p1);
    scatter2<19, ODD, S, 0, false, ZW, FAST, Off>(kp, f, st, f0, f1);
    scatter2<NS, ODD, S, D0, R32, ZW, FAST, Off>(kp, phi, st, p0, p1);
}

// Two x-adjacent nodes per thread (nx even): paired population accesses, see
// lbm_aa2.cuh.  Same arithmetic per node as bgk_step_kernel.  On odd steps
// the rows away from the z walls (uniform per block) take a body without the
// wall selects.
template <bool ODD, bool SAVE, typename S, int SL, typename Off = unsigned>
__global__ void __launch_bounds__(128, std::is_same<S, float>::value ? LBM_STEP2_MINB : LBM_STEP2_MINB16) bgk_step2_kernel(KParams kp, S* __restrict__ f,
                                                                    S* __restrict__ phi,
                                                                    float* __restrict__ save) {
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const Stencil2 st = make_stencil2(kp, x, blockIdx.y, blockIdx.z);
    const int z = blockIdx.z;
    const bool zwall = ODD && (!LBM_BGK_ZSPLIT ||
                               (!(kp.flags & LBM_FLAG_PERIODIC_Z) && (z == 0 || z == kp.nz - 1)));
    if (!ODD) bgk_step2_body<ODD, SAVE, S, SL, false, false, Off>(kp, f, phi, save, st);
    else if (LBM_BGK_FAST && block_interior2(kp))
        bgk_step2_body<ODD, SAVE, S, SL, false, true, Off>(kp, f, phi, save, st);
    else if (!zwall) bgk_step2_body<ODD, SAVE, S, SL, false, false, Off>(kp, f, phi, save, st);
    else bgk_step2_body<ODD, SAVE, S, SL, true, false, Off>(kp, f, phi, save, st);
}

#ifndef LBM_BGK_QUAD
#define LBM_BGK_QUAD 1
#endif
#ifndef LBM_STEP4_MINB
#define LBM_STEP4_MINB 3
#endif

// Even steps with 16-bit storage and nx a multiple of 4: four x-adjacent
// nodes per thread, each population row moved as one aligned 8-byte word
// (a warp reads and writes 256-byte row segments, as the FP32 pair kernel
// does, against 128 for 16-bit pairs).  Even steps are local (slot i of node
// n is read, slot opp(i) of the same node written), so the words need no
// shifting; the four nodes are unpacked, collided and packed back one at a
// time.  Same arithmetic per node as bgk_step_kernel.  Odd steps stay with
// bgk_step2_kernel: there the x-shifted rows of a packed quad need shuffles
// and byte permutes and measured slower than the paired form.
struct BgkQuadCollide {
    template <int SL, typename S>
    static __device__ __forceinline__ void run(const KParams& kp, float (&f)[19],
                                               float (&p)[ScalarLat<SL>::NS]) {
        collide_bgk<true, SL>(kp, f, p);
    }
};

template <typename S, int SL, typename Off = unsigned>
__global__ void __launch_bounds__(128, LBM_STEP4_MINB) bgk_even4_kernel(KParams kp, S* __restrict__ f,
                                                                       S* __restrict__ phi) {
    even4_body<19, SL, S, Off, BgkQuadCollide>(kp, f, phi);
}

template <typename S, int SL, typename Off>
static cudaError_t launch_bgk_off(const KParams& kp, bool odd, S* f, S* phi, float* save,
                                  cudaStream_t st) {
    if constexpr (LBM_BGK_QUAD && !std::is_same<S, float>::value) {
        if (!odd && !save && kp.nx % 4 == 0 && !(kp.flags & LBM_FLAG_ONE_NODE)) {
            dim3 block(128), grid((kp.nx / 4 + 127) / 128, kp.ny, kp.nz);
            bgk_even4_kernel<S, SL, Off><<<grid, block, 0, st>>>(kp, f, phi);
            return cudaGetLastError();
        }
    }
    if constexpr (LBM_BGK_PAIR) if (kp.nx % 2 == 0 && !(kp.flags & LBM_FLAG_ONE_NODE)) {
        dim3 block(128), grid((kp.nx / 2 + 127) / 128, kp.ny, kp.nz);
        if (save) {
            if constexpr (std::is_same<Off, unsigned>::value) {
                if (odd) bgk_step2_kernel<true, true, S, SL><<<grid, block, 0, st>>>(kp, f, phi, save);
                else bgk_step2_kernel<false, true, S, SL><<<grid, block, 0, st>>>(kp, f, phi, save);
            } else {
                return cudaErrorInvalidValue;   // saved steps need (Q + NS) N < 2^32
            }
        } else {
            if (odd) bgk_step2_kernel<true, false, S, SL, Off><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
            else bgk_step2_kernel<false, false, S, SL, Off><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
        }
        return cudaGetLastError();
    }
    dim3 block(128), grid((kp.nx + 127) / 128, kp.ny, kp.nz);
    if (save) {
        if constexpr (std::is_same<Off, unsigned>::value) {
            if (odd) bgk_step_kernel<true, true, S, SL><<<grid, block, 0, st>>>(kp, f, phi, save);
            else bgk_step_kernel<false, true, S, SL><<<grid, block, 0, st>>>(kp, f, phi, save);
        } else {
            return cudaErrorInvalidValue;
        }
    } else {
        if (odd) bgk_step_kernel<true, false, S, SL, Off><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
        else bgk_step_kernel<false, false, S, SL, Off><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
    }
    return cudaGetLastError();
}

// 32-bit element offsets unless (Q + NS) N >= 2^32 (KParams::wide).
template <typename S, int SL>
static cudaError_t launch_bgk_typed(const KParams& kp, bool odd, S* f, S* phi, float* save,
                                   cudaStream_t st) {
    if (kp.wide) return launch_bgk_off<S, SL, size_t>(kp, odd, f, phi, save, st);
    return launch_bgk_off<S, SL, unsigned>(kp, odd, f, phi, save, st);
}

template <int SL>
static cudaError_t launch_bgk_sl(const KParams& kp, int storage, bool odd, void* f, void* phi,
                                 float* save, cudaStream_t st) {
    switch (storage) {
        case LBM_FP32: return launch_bgk_typed<float, SL>(kp, odd, (float*)f, (float*)phi, save, st);
        case LBM_FP16S: return launch_bgk_typed<__half, SL>(kp, odd, (__half*)f, (__half*)phi, save, st);
        case LBM_BF16S:
            return launch_bgk_typed<__nv_bfloat16, SL>(kp, odd, (__nv_bfloat16*)f,
                                                       (__nv_bfloat16*)phi, save, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_bgk_step(const KParams& kp, int storage, int scalar, bool odd, void* f,
                            void* phi, float* save, cudaStream_t st) {
    if (scalar == LBM_SCALAR_Q7) return launch_bgk_sl<7>(kp, storage, odd, f, phi, save, st);
    if (scalar == LBM_SCALAR_Q6) return launch_bgk_sl<6>(kp, storage, odd, f, phi, save, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbmgpu
