// lbm_quad.cuh -- even AA steps of 16-bit storage on four x-adjacent nodes
// per thread.
//
// Even steps are local: slot i of node n is read and slot opp(i) of the same
// node written (lbm_common.cuh).  With nx a multiple of 4, thread t owns the
// nodes x = 4t .. 4t + 3 of a row and moves every population row as one
// aligned 8-byte word, so a warp reads and writes 256-byte row segments (as
// the FP32 pair kernel does) instead of the 64 bytes of one 2-byte element
// per thread.  The words stay packed in registers (two 16-bit values per
// 32-bit half); the four nodes are unpacked, collided and packed back one at
// a time, so only one node's populations are live as floats.  Same
// arithmetic per node as the one-node kernels.
#pragma once

#include "lbm_common.cuh"

namespace lbmgpu {

// Two 16-bit values packed in a 32-bit word: the lower node in the low half
// (hi = 0), the upper in the high half (hi = 1).
template <typename S> struct Half16;
template <> struct Half16<__half> {
    static __device__ __forceinline__ float get(unsigned w, int hi) {
        return __half2float(__ushort_as_half((unsigned short)(hi ? w >> 16 : w & 0xffffu)));
    }
    static __device__ __forceinline__ unsigned bits(float v) {
        return __half_as_ushort(__float2half_rn(v));
    }
};
template <> struct Half16<__nv_bfloat16> {
    static __device__ __forceinline__ float get(unsigned w, int hi) {
        return __uint_as_float(hi ? w & 0xffff0000u : w << 16);   // exact widening
    }
    static __device__ __forceinline__ unsigned bits(float v) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
};
// w with its low (hi = 0) or high (hi = 1) half replaced by the low half of b.
__device__ __forceinline__ unsigned put16(unsigned w, unsigned b, int hi) {
    return __byte_perm(w, b, hi ? 0x5410 : 0x3254);
}

// Packed words of NODES (2 or 4) x-adjacent 16-bit values, and their rest
// row counterpart (FP32).
template <int NODES> struct Packed;
template <> struct Packed<2> {
    using W = unsigned;
    using R = float2;
    static __device__ __forceinline__ unsigned& half(W& w, int j) { return w; }
    static __device__ __forceinline__ float& rest(R& r, int j) { return j == 0 ? r.x : r.y; }
    static __device__ __forceinline__ W zero() { return 0u; }
    static __device__ __forceinline__ R rzero() { return make_float2(0.0f, 0.0f); }
};
template <> struct Packed<4> {
    using W = uint2;
    using R = float4;
    static __device__ __forceinline__ unsigned& half(W& w, int j) { return j < 2 ? w.x : w.y; }
    static __device__ __forceinline__ float& rest(R& r, int j) {
        return j == 0 ? r.x : j == 1 ? r.y : j == 2 ? r.z : r.w;
    }
    static __device__ __forceinline__ W zero() { return make_uint2(0u, 0u); }
    static __device__ __forceinline__ R rzero() { return make_float4(0.0f, 0.0f, 0.0f, 0.0f); }
};

// The even step of the NODES nodes of this thread (grid: nx / NODES threads
// along x, rows y = blockIdx.y, z = blockIdx.z; nx a multiple of NODES).  Q
// fluid populations, the scalar lattice SL; Collide::run(kp, f, p) collides
// one node in storage units.  R32: the scalar's rest population lives in the
// FP32 rest row (rest_row), moved as one float2 / float4 per thread.
template <int Q, int SL, typename S, typename Off, typename Collide, int NODES = 4>
__device__ __forceinline__ void even4_body(const KParams& kp, S* __restrict__ f,
                                           S* __restrict__ phi) {
    using P = Packed<NODES>;
    using W = typename P::W;
    using R = typename P::R;
    const unsigned x = NODES * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= (unsigned)kp.nx) return;
    constexpr int NS = ScalarLat<SL>::NS, D0 = ScalarLat<SL>::D0;
    constexpr bool R32 = rest32<S, SL>();
    const unsigned N = kp.N;
    const unsigned n = blockIdx.z * kp.nxny + blockIdx.y * kp.nx + x;
    W* __restrict__ fw = reinterpret_cast<W*>(f);
    W* __restrict__ pw = reinterpret_cast<W*>(phi);
    R* __restrict__ rest = reinterpret_cast<R*>(rest_row(phi, NS, N) + n);
    W wf[Q], wp[NS];
    R r = P::rzero();
    // the NODES elements of each word, checked in the debug build
    auto ok = [&](const S* a, Off o, int rows) {
        return LBM_IN(kp, LBM_SITE_QUAD, a, a + o, NODES, (size_t)rows * N);
    };
    const bool rest_ok = !R32 || LBM_IN(kp, LBM_SITE_QUAD, rest_row(phi, NS, N),
                                        rest_row(phi, NS, N) + n, NODES, N);
    constexpr int SH = NODES == 4 ? 2 : 1;   // element offset -> word offset
#pragma unroll
    for (int i = 0; i < Q; ++i)
        wf[i] = ok(f, (Off)i * N + n, Q) ? ld_pop(fw + (((Off)i * N + n) >> SH)) : P::zero();
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        if (R32 && k == 0) {
            if (rest_ok) r = ld_pop(rest);
        } else {
            wp[k] = ok(phi, (Off)k * N + n, NS) ? ld_pop(pw + (((Off)k * N + n) >> SH)) : P::zero();
        }
    }
    const bool collide = !(kp.flags & LBM_FLAG_NO_COLLIDE);
#pragma unroll
    for (int j = 0; j < NODES; ++j) {   // node x + j: 32-bit half j / 2, 16-bit half j % 2
        float fv[Q], pv[NS];
#pragma unroll
        for (int i = 0; i < Q; ++i) fv[i] = Half16<S>::get(P::half(wf[i], j), j & 1);
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (R32 && k == 0) pv[0] = P::rest(r, j);
            else pv[k] = Half16<S>::get(P::half(wp[k], j), j & 1);
        }
        if (collide) Collide::template run<SL, S>(kp, fv, pv);
        if constexpr (R32) feed_rest<S>(pv);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            unsigned& w = P::half(wf[i], j);
            w = put16(w, Half16<S>::bits(fv[i]), j & 1);
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (R32 && k == 0) {
                P::rest(r, j) = pv[0];
            } else {
                unsigned& w = P::half(wp[k], j);
                w = put16(w, Half16<S>::bits(pv[k]), j & 1);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (ok(f, (Off)opp(i) * N + n, Q)) st_pop(fw + (((Off)opp(i) * N + n) >> SH), wf[i]);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        if (R32 && k == 0) {
            if (rest_ok) st_pop(rest, r);
        } else if (ok(phi, (Off)(opp(k + D0) - D0) * N + n, NS)) {
            st_pop(pw + (((Off)(opp(k + D0) - D0) * N + n) >> SH), wp[k]);
        }
    }
}

}  // namespace lbmgpu
