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
#include "lbm_quad.cuh"

namespace lbmgpu {

// Minimum resident blocks per SM for the register allocator: the D3Q27 FCM
// scalar holds more live values, so its instantiation gets its own setting,
// per parity: odd steps 3 (168 registers, 36 bytes of spills; with 32-bit
// offsets on both parities 3 measured 14.1 G node updates/s against 11.9
// for 2 and 11.3 for 4), even steps 4 (below).
#ifndef LBM_Q27_MINB
#define LBM_Q27_MINB 3
#endif
#ifndef LBM_Q27_MINB_EVEN
#define LBM_Q27_MINB_EVEN 4
#endif
// Even steps of the D3Q27-scalar instantiation take 64-bit element offsets
// on every box: with 32-bit offsets the compiler keeps the scalar's 27
// offsets of the first read live across the fluid collision for the second
// read (216 bytes of spills at 128 registers), with 64-bit ones it recomputes
// them and fits 128 registers without spills (4 blocks per SM): 4.65 -> 4.33
// ms per even step at 2048x128x256 (FP32).  Odd steps keep 32-bit offsets at
// 168 registers (36 bytes of spills): their 64-bit form took 5.35 ms against
// 4.88, and a spill-free 32-bit form whose second read recomputes its
// neighbour offsets from an opaque copy of the stencil 5.20.
#ifndef LBM_Q27_WIDE_EVEN
#define LBM_Q27_WIDE_EVEN 1
#endif
#ifndef LBM_CUM_MINB
#define LBM_CUM_MINB LBM_STEP_MINB
#endif
// Even steps of the D3Q7-scalar instantiation: 64-bit element offsets on
// every box and 6 resident blocks (80 registers).  With 64-bit offsets the
// compiler walks each array by a pointer and a row stride instead of keeping
// 34 row offsets, so the kernel fits 80 registers (FP32 without spills, 16
// bits with 24 bytes) where the 32-bit form spills 216 bytes; at 2048x128x256
// the even step took 2.85 -> 2.75 ms (FP32), 2.16 -> 2.12 (FP16), 2.18 ->
// 2.13 (BF16).  7 and 8 blocks (72, 64 registers) and the 64-bit form at 4
// blocks measured slower; odd steps, whose neighbour offsets are the live
// values, keep 32-bit offsets and 4 blocks (5 blocks: 208 bytes of spills,
// 2.22 -> 2.69 ms per FP16 odd step).
#ifndef LBM_CUM_MINB_EVEN
#define LBM_CUM_MINB_EVEN 6
#endif
#ifndef LBM_CUM_WIDE_EVEN
#define LBM_CUM_WIDE_EVEN 1
#endif
#ifndef LBM_CUM_WSPLIT
#define LBM_CUM_WSPLIT 1
#endif
// Odd steps of blocks with no node at a face of the box read and write at
// block-uniform offsets from the node (block_no_face below): 2.26 -> 2.20 ms
// per odd step at 2048x128x256 (FP16), 2.31 -> 2.27 (BF16), 3.04 -> 3.01
// (FP32).  The same form in the paired BGK kernel's wall-free body measured
// slower (FP16 odd 1.54 -> 1.59 ms), and as a second odd body of the D3Q27
// FCM instantiation no faster (FP32 4.90 -> 4.89 ms, FP16 4.04 -> 4.11, 36 ->
// 92 bytes of spills in FP32); neither was adopted.  Running the blocks
// away from every face as a kernel of their own (a compact grid, the
// block-uniform body alone, 64-bit offsets: 80 registers without spills, 6
// blocks per SM) and the face blocks as a second launch (enumerated on a 1-D
// grid) measured FP32 odd steps 3.01 -> 2.97 ms but FP16 2.20 -> 2.43 and
// BF16 2.27 -> 2.43, and was not adopted either.
#ifndef LBM_CUM_NOFACE
#define LBM_CUM_NOFACE 1
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
                save_pop(kp, save, 54, 27 + k, n, s16 ? phi_canonical(kp, pv[k], w27(k)) : pv[k]);
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

// Odd steps of a block none of whose nodes has a neighbour across a face of
// the box (block_no_face): no wall and no periodic wrap is involved, so the
// element offset of population k's source (row opp(d), node n - c_d) is n +
// ((opp(d) - D0) N - c_dx - c_dy nx - c_dz nx ny), and of its target (row k,
// node n + c_d) n + (k N + c_dx + c_dy nx + c_dz nx ny): the brackets are the
// same for every thread of the block.  Offsets are formed modulo 2^32 (or
// 2^64) with Off; the sums land inside the arrays.
__device__ __forceinline__ bool block_no_face(const KParams& kp) {
    const int x0 = blockIdx.x * blockDim.x, y = blockIdx.y, z = blockIdx.z;
    return x0 >= 1 && x0 + (int)blockDim.x <= kp.nx - 1 && y >= 1 && y <= kp.ny - 2 && z >= 1 &&
           z <= kp.nz - 2;
}
template <typename Off>
__device__ __forceinline__ Off shift_of(const KParams& kp, int d) {
    return (Off)(long long)(cx27(d) + cy27(d) * kp.nx + cz27(d) * (long long)kp.nxny);
}
template <int Q, typename S, int D0 = 0, bool R32 = false, typename Off = unsigned>
__device__ __forceinline__ void gather_no_face(const KParams& kp, const S* __restrict__ a,
                                               unsigned n, float (&v)[Q]) {
    const unsigned N = kp.N;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int d = k + D0;
        if (R32 && d == 0) {
            const float* r = rest_row(a, Q, N);
            v[k] = LBM_IN(kp, LBM_SITE_GATHER, r, r + n, 1, N) ? ld_pop(r + n) : 0.0f;
            continue;
        }
        const Off o = d == 0 ? (Off)k * N : (Off)(opp(d) - D0) * N - shift_of<Off>(kp, d);
        const Off e = (Off)n + o;
        v[k] = LBM_IN(kp, LBM_SITE_GATHER, a, a + e, 1, (size_t)Q * N) ? Store<S>::ld(a + e) : 0.0f;
    }
}
template <int Q, typename S, int D0 = 0, bool R32 = false, typename Off = unsigned>
__device__ __forceinline__ void scatter_no_face(const KParams& kp, S* __restrict__ a, unsigned n,
                                                const float (&v)[Q]) {
    const unsigned N = kp.N;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int d = k + D0;
        if (R32 && d == 0) {
            float* r = rest_row(a, Q, N);
            if (LBM_IN(kp, LBM_SITE_SCATTER, r, r + n, 1, N)) st_pop(r + n, v[k]);
            continue;
        }
        const Off o = d == 0 ? (Off)k * N : (Off)k * N + shift_of<Off>(kp, d);
        const Off e = (Off)n + o;
        if (LBM_IN(kp, LBM_SITE_SCATTER, a, a + e, 1, (size_t)Q * N)) Store<S>::st(a + e, v[k]);
    }
}

template <bool ODD, bool SAVE, typename S, int SL, bool W, typename Off, bool NOFACE = false>
__device__ __forceinline__ void cumulant_step_body(const KParams& kp, S* __restrict__ f,
                                                   S* __restrict__ phi, float* __restrict__ save,
                                                   const Stencil& st) {
    const unsigned n = st.n;
    constexpr int NS = ScalarLat<SL>::NS;
    constexpr bool R32 = rest32<S, SL>();
    float fv[27], pv[NS];
    if constexpr (NOFACE) {
        gather_no_face<27, S, 0, false, Off>(kp, f, n, fv);
        gather_no_face<NS, S, 0, R32, Off>(kp, phi, n, pv);
    } else {
        gather<27, ODD, S, 0, false, W, Off>(kp, f, st, fv);
        gather<NS, ODD, S, 0, R32, W, Off>(kp, phi, st, pv);
    }
    constexpr bool s16 = !std::is_same<S, float>::value;   // populations in storage units
    constexpr bool fold = s16 && SL == 7;                  // the collision applies the scales
    if (SAVE) {
#pragma unroll
        for (int i = 0; i < 27; ++i)
            save_pop(kp, save, 27 + NS, i, n, s16 ? fv[i] * kp.isf : fv[i]);
#pragma unroll
        for (int k = 0; k < NS; ++k)
            save_pop(kp, save, 27 + NS, 27 + k, n,
                     s16 ? phi_canonical(kp, pv[k], ScalarLat<SL>::w(k)) : pv[k]);
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
    if constexpr (NOFACE) {
        scatter_no_face<27, S, 0, false, Off>(kp, f, n, fv);
        scatter_no_face<NS, S, 0, R32, Off>(kp, phi, n, pv);
    } else {
        scatter<27, ODD, S, 0, false, W, Off>(kp, f, st, fv);
        scatter<NS, ODD, S, 0, R32, W, Off>(kp, phi, st, pv);
    }
}

// One node per thread.  On odd steps the blocks with no wall neighbour
// (uniform per block) take a body without the wall selects (D3Q7 scalar:
// measured 0.6-0.9 % faster; with the D3Q27 scalar the second body costs
// registers and was 4 % slower, so that instantiation keeps one body).
template <bool ODD, bool SAVE, typename S, int SL, typename Off = unsigned>
__global__ void __launch_bounds__(128, SL == 27 ? (ODD || SAVE ? LBM_Q27_MINB : LBM_Q27_MINB_EVEN)
                                                : (ODD || SAVE ? LBM_CUM_MINB : LBM_CUM_MINB_EVEN))
    cumulant_step_kernel(KParams kp, S* __restrict__ f,
                                                            S* __restrict__ phi,
                                                            float* __restrict__ save) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const Stencil st = make_stencil(kp, x, blockIdx.y, blockIdx.z);
    if constexpr (SL == 27) {
        cumulant_fcm_step_body<ODD, SAVE, S, true, Off>(kp, f, phi, save, st);
    } else {
        if (!ODD)
            cumulant_step_body<ODD, SAVE, S, SL, false, Off>(kp, f, phi, save, st);
        else if (LBM_CUM_NOFACE && block_no_face(kp))
            cumulant_step_body<ODD, SAVE, S, SL, false, Off, true>(kp, f, phi, save, st);
        else if (!LBM_CUM_NOFACE && LBM_CUM_WSPLIT && block_interior(kp))
            cumulant_step_body<ODD, SAVE, S, SL, false, Off>(kp, f, phi, save, st);
        else
            cumulant_step_body<ODD, SAVE, S, SL, true, Off>(kp, f, phi, save, st);
    }
}

// Even steps of 16-bit storage with the D3Q7 scalar and nx a multiple of 4:
// four nodes per thread on packed 8-byte words (lbm_quad.cuh), 168 registers
// (72 bytes of spills): 2.14 -> 1.90 ms per even step at 2048x128x256 (FP16),
// 2.15 -> 1.92 (BF16).  Two nodes per thread on 4-byte words measured 2.12
// (no spills at 168 registers) and 2.16 (128 registers), four nodes at 255
// registers 2.20.  Odd steps keep the one-node kernel: a four-node odd form
// (aligned words of every row, the x-shifted rows assembled by a 32-bit
// shuffle and a byte permute, the warp-edge elements loaded and stored by
// the edge lanes; bit-identical streaming) took 3.12 ms against 2.27,
// issuing 916 instructions per node against 865 (unpacking, repacking and
// the edge stores cost more than the loads they save) at 50 % issue
// activity with 12 warps per SM.
#ifndef LBM_CUM_QUAD
#define LBM_CUM_QUAD 1
#endif
#ifndef LBM_CUM_QUAD_MINB
#define LBM_CUM_QUAD_MINB 3
#endif
#ifndef LBM_CUM_QUAD_OFF
#define LBM_CUM_QUAD_OFF size_t
#endif
#ifndef LBM_CUM_QUAD_NODES
#define LBM_CUM_QUAD_NODES 4
#endif
struct CumulantQuadCollide {
    template <int SL, typename S>
    static __device__ __forceinline__ void run(const KParams& kp, float (&f)[27],
                                               float (&p)[ScalarLat<SL>::NS]) {
        collide_cumulant<SL, true>(kp, f, p);   // D3Q7: the collision applies the scales
    }
};

template <typename S, typename Off>
__global__ void __launch_bounds__(128, LBM_CUM_QUAD_MINB)
    cumulant_even4_kernel(KParams kp, S* __restrict__ f, S* __restrict__ phi) {
    even4_body<27, 7, S, Off, CumulantQuadCollide, LBM_CUM_QUAD_NODES>(kp, f, phi);
}

template <typename S, int SL>
static cudaError_t launch_cumulant_typed(const KParams& kp, bool odd, S* f, S* phi, float* save,
                                        cudaStream_t st) {
    if constexpr (LBM_CUM_QUAD && SL == 7 && !std::is_same<S, float>::value) {
        constexpr int QN = LBM_CUM_QUAD_NODES;
        if (!odd && !save && kp.nx % QN == 0 && !(kp.flags & LBM_FLAG_ONE_NODE)) {
            dim3 block(128), grid((kp.nx / QN + 127) / 128, kp.ny, kp.nz);
            if (kp.wide)
                cumulant_even4_kernel<S, size_t><<<grid, block, 0, st>>>(kp, f, phi);
            else
                cumulant_even4_kernel<S, LBM_CUM_QUAD_OFF><<<grid, block, 0, st>>>(kp, f, phi);
            return cudaGetLastError();
        }
    }
    dim3 block(128), grid((kp.nx + 127) / 128, kp.ny, kp.nz);
    // even steps with 64-bit offsets on every box
    constexpr bool wide_even = SL == 27 ? LBM_Q27_WIDE_EVEN : LBM_CUM_WIDE_EVEN;
    if (kp.wide) {   // (Q + NS) N >= 2^32: 64-bit element offsets; no saved steps
        if (save) return cudaErrorInvalidValue;
        if (odd) cumulant_step_kernel<true, false, S, SL, size_t><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
        else cumulant_step_kernel<false, false, S, SL, size_t><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
        return cudaGetLastError();
    }
    if (save) {
        if (odd) cumulant_step_kernel<true, true, S, SL><<<grid, block, 0, st>>>(kp, f, phi, save);
        else cumulant_step_kernel<false, true, S, SL><<<grid, block, 0, st>>>(kp, f, phi, save);
    } else if (odd) {
        cumulant_step_kernel<true, false, S, SL><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
    } else if constexpr (wide_even) {
        cumulant_step_kernel<false, false, S, SL, size_t><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
    } else {
        cumulant_step_kernel<false, false, S, SL><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
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
