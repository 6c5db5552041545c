// lbm_aa2.cuh -- AA gather / scatter for two x-adjacent nodes per thread.
//
// Thread t of a row segment owns the nodes x = 2t and x + 1 (nx even) and
// moves each population row as aligned pairs (8 bytes in FP32, 4 bytes in
// FP16 / BF16), so a warp reads or writes 64 consecutive nodes of a row with
// one request per population.  On odd steps the populations with c_x != 0
// come from (go to) x -+ 1: the pair is read aligned and the element that
// belongs to the neighbouring thread is exchanged with a warp shuffle; the
// first and last active lanes of a warp load / store the one element that
// lies in the neighbouring warp's range themselves.
//
// In-place safety: for every population row, each element is loaded and
// stored by the same thread within a step (the AA property of
// lbm_common.cuh holds per element).  The only exception is the aligned pair
// load of a boundary lane, whose half that belongs to the next warp is read
// but never used.
#pragma once

#include "lbm_common.cuh"

namespace lbmgpu {

template <typename S> struct PairIO;
template <> struct PairIO<float> {
    static __device__ __forceinline__ void ld(const float* p, float& a, float& b) {
        const float2 v = ld_pop(reinterpret_cast<const float2*>(p));
        a = v.x; b = v.y;
    }
    static __device__ __forceinline__ void st(float* p, float a, float b) {
        st_pop(reinterpret_cast<float2*>(p), make_float2(a, b));
    }
    static __device__ __forceinline__ void rnd(float& a, float& b) {}
};
template <> struct PairIO<__half> {
    static __device__ __forceinline__ void ld(const __half* p, float& a, float& b) {
        const __half2 v = ld_pop(reinterpret_cast<const __half2*>(p));
        const float2 f = __half22float2(v);
        a = f.x; b = f.y;
    }
    static __device__ __forceinline__ void st(__half* p, float a, float b) {
        st_pop(reinterpret_cast<__half2*>(p), __floats2half2_rn(a, b));
    }
    static __device__ __forceinline__ void rnd(float& a, float& b) {
        const float2 f = __half22float2(__floats2half2_rn(a, b));
        a = f.x; b = f.y;
    }
};
template <> struct PairIO<__nv_bfloat16> {
    static __device__ __forceinline__ void ld(const __nv_bfloat16* p, float& a, float& b) {
        const __nv_bfloat162 v = ld_pop(reinterpret_cast<const __nv_bfloat162*>(p));
        const float2 f = __bfloat1622float2(v);
        a = f.x; b = f.y;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float a, float b) {
        st_pop(reinterpret_cast<__nv_bfloat162*>(p), __floats2bfloat162_rn(a, b));
    }
    static __device__ __forceinline__ void rnd(float& a, float& b) {
        const float2 f = __bfloat1622float2(__floats2bfloat162_rn(a, b));
        a = f.x; b = f.y;
    }
};

// feed_rest (lbm_common.cuh) for a node pair, with paired conversions.
template <typename S, int NS>
__device__ __forceinline__ void feed_rest2(float (&p0)[NS], float (&p1)[NS]) {
    float e0 = 0.0f, e1 = 0.0f;
#pragma unroll
    for (int k = 1; k < NS; ++k) {
        float r0 = p0[k], r1 = p1[k];
        PairIO<S>::rnd(r0, r1);
        e0 += p0[k] - r0;
        e1 += p1[k] - r1;
        p0[k] = r0;
        p1[k] = r1;
    }
    p0[0] += e0;
    p1[0] += e1;
}

// Neighbourhood of a node pair (x, x + 1), x even.
struct Stencil2 {
    unsigned n;         // node x
    unsigned zr[3];     // (z + dz) * nx * ny, dz = -1, 0, 1
    unsigned yr[3];     // (y + dy) * nx,      dy = -1, 0, 1
    unsigned x, xm, xp2;// x, x - 1 (wrapped), x + 2 (wrapped)
    bool zo[3];         // row z + dz in the fluid (or wrapped)
    bool xmo, xp2o;     // x - 1, x + 2 in the fluid (or wrapped)
    bool active;        // x < nx
    bool left, right;   // this lane loads / stores across the warp's left / right edge
};

__device__ __forceinline__ Stencil2 make_stencil2(const KParams& kp, int x, int y, int z) {
    Stencil2 s;
    const bool px = (kp.flags & LBM_FLAG_PERIODIC_X) != 0;
    const bool pz = (kp.flags & LBM_FLAG_PERIODIC_Z) != 0;
    const int ym = y == 0 ? kp.ny - 1 : y - 1, yp = y == kp.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? kp.nz - 1 : z - 1, zp = z == kp.nz - 1 ? 0 : z + 1;
    s.yr[0] = (unsigned)ym * kp.nx; s.yr[1] = (unsigned)y * kp.nx; s.yr[2] = (unsigned)yp * kp.nx;
    s.zr[0] = (unsigned)zm * kp.nxny; s.zr[1] = (unsigned)z * kp.nxny; s.zr[2] = (unsigned)zp * kp.nxny;
    s.zo[0] = z > 0 || pz; s.zo[1] = true; s.zo[2] = z < kp.nz - 1 || pz;
    s.active = x < kp.nx;
    s.x = (unsigned)x;
    s.xm = (unsigned)(x == 0 ? kp.nx - 1 : x - 1);
    s.xp2 = (unsigned)(x + 2 >= kp.nx ? x + 2 - kp.nx : x + 2);
    s.xmo = x > 0 || px;
    s.xp2o = x + 2 < kp.nx || px;
    const int lane = threadIdx.x & 31;
    s.left = lane == 0;
    s.right = lane == 31 || x + 2 >= kp.nx;
    s.n = s.zr[1] + s.yr[1] + (unsigned)x;
    return s;
}

// True when every node pair of this block is active and has all its
// neighbours inside the box (x - 1 >= 0, x + 2 <= nx - 1, 1 <= z <= nz - 2):
// the condition of the FAST accesses below, uniform over the block.
__device__ __forceinline__ bool block_interior2(const KParams& kp) {
    const int x0 = 2 * blockIdx.x * blockDim.x, z = blockIdx.z;
    return x0 >= 1 && x0 + 2 * (int)blockDim.x <= kp.nx - 1 && z >= 1 && z <= kp.nz - 2;
}

// The gather runs in three phases so that no shuffle waits on a load issued
// after it: (1) every aligned pair load, (2) the edge lanes' single-element
// loads, predicated, (3) the shuffles that hand the shifted element across.
// A z wall (uniform over the block) turns a direction into a bounce-back from
// the node's own slot, selected without branching.
// R32: population 0 (direction 0) lives in the FP32 rest row (rest_row).
// ZW: the node pair may lie next to a z wall; false for the z-interior rows,
// which then skip the wall selects (every z neighbour is in the fluid).
// FAST (odd steps of blocks whose every node has all its neighbours in the
// fluid and every lane active): the x-shifted populations are read and
// written as two single elements per thread, x + dx and x + 1 + dx, instead
// of an aligned pair, a shuffle and the warp-edge element.  Each node still
// reads and writes exactly the elements it owns in the AA step, so the
// in-place update stays race-free.
template <int Q, bool ODD, typename S, int D0 = 0, bool R32 = false, bool ZW = true,
          bool FAST = false, typename Off = unsigned>
__device__ __forceinline__ void gather2(const KParams& kp, const S* __restrict__ a,
                                        const Stencil2& st, float (&v0)[Q], float (&v1)[Q]) {
    const unsigned N = kp.N;
    constexpr bool ZWe = ZW && !FAST;
    float P0[Q], P1[Q], E[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int i = k + D0;       // direction; population k lives in row k
        if (R32 && i == 0) {
            P0[k] = 0.0f; P1[k] = 0.0f;
            const float* r = rest_row(a, Q, N);
            if (st.active && LBM_IN(kp, LBM_SITE_PAIR_LOAD, r, r + st.n, 2, N))
                PairIO<float>::ld(r + st.n, P0[k], P1[k]);
            continue;
        }
        Off off = (Off)k * N + st.n;
        if (ODD && i != 0) {
            const int dx = -cx27(i), dy = -cy27(i), dz = -cz27(i);
            const Off row = (Off)(opp(i) - D0) * N + st.zr[dz + 1] + st.yr[dy + 1];
            if (FAST && dx != 0) {
                const Off e = row + st.x + (Off)dx;
                if (LBM_IN(kp, LBM_SITE_PAIR_LOAD, a, a + e, 2, (size_t)Q * N)) {
                    P0[k] = Store<S>::ld(a + e);
                    P1[k] = Store<S>::ld(a + e + 1);
                } else {
                    P0[k] = 0.0f; P1[k] = 0.0f;
                }
                continue;
            }
            off = (!ZWe || st.zo[dz + 1]) ? row + st.x : off;
        }
        P0[k] = 0.0f; P1[k] = 0.0f;
        if (st.active && LBM_IN(kp, LBM_SITE_PAIR_LOAD, a, a + off, 2, (size_t)Q * N))
            PairIO<S>::ld(a + off, P0[k], P1[k]);
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int i = k + D0;
        E[k] = 0.0f;
        const int dx = -cx27(i), dy = -cy27(i), dz = -cz27(i);
        if (ODD && !FAST && i != 0 && dx != 0) {
            const Off row = (Off)(opp(i) - D0) * N + st.zr[dz + 1] + st.yr[dy + 1];
            const Off own = (Off)k * N + st.n;
            Off off;
            bool need;
            if (dx < 0) { need = st.left; off = st.xmo ? row + st.xm : own; }
            else { need = st.right; off = st.xp2o ? row + st.xp2 : own + 1; }
            need = need && st.active && (!ZWe || st.zo[dz + 1]);
            if (need && LBM_IN(kp, LBM_SITE_PAIR_LOAD, a, a + off, 1, (size_t)Q * N))
                E[k] = Store<S>::ld(a + off);
        }
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int i = k + D0;
        const int dx = -cx27(i), dz = -cz27(i);
        v0[k] = P0[k]; v1[k] = P1[k];
        if (ODD && !FAST && i != 0 && dx != 0) {
            const bool in = !ZWe || st.zo[dz + 1];
            if (dx < 0) {
                // node x needs element x - 1, node x + 1 needs element x
                const float e = __shfl_up_sync(0xffffffffu, P1[k], 1);
                v0[k] = in ? (st.left ? E[k] : e) : P0[k];
                v1[k] = in ? P0[k] : P1[k];
            } else {
                // node x needs element x + 1, node x + 1 needs element x + 2
                const float e = __shfl_down_sync(0xffffffffu, P0[k], 1);
                v0[k] = in ? P1[k] : P0[k];
                v1[k] = in ? (st.right ? E[k] : e) : P1[k];
            }
        }
    }
}

// The scatter first exchanges the shifted elements, then issues every store
// under a predicate (pair stores for the interior lanes, single-element
// stores for the edge lanes, pair stores into the own slots at a z wall).
template <int Q, bool ODD, typename S, int D0 = 0, bool R32 = false, bool ZW = true,
          bool FAST = false, typename Off = unsigned>
__device__ __forceinline__ void scatter2(const KParams& kp, S* __restrict__ a, const Stencil2& st,
                                         const float (&v0)[Q], const float (&v1)[Q]) {
    const unsigned N = kp.N;
    constexpr bool ZWe = ZW && !FAST;
    float X[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int i = k + D0;
        const int dx = cx27(i);
        X[k] = 0.0f;
        if (ODD && !FAST && i != 0 && dx > 0) X[k] = __shfl_up_sync(0xffffffffu, v1[k], 1);
        if (ODD && !FAST && i != 0 && dx < 0) X[k] = __shfl_down_sync(0xffffffffu, v0[k], 1);
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int i = k + D0;
        const int dx = cx27(i), dy = cy27(i), dz = cz27(i);
        if (R32 && i == 0) {
            float* r = rest_row(a, Q, N);
            if (st.active && LBM_IN(kp, LBM_SITE_PAIR_STORE, r, r + st.n, 2, N))
                PairIO<float>::st(r + st.n, v0[k], v1[k]);
            continue;
        }
        const Off own = (Off)(opp(i) - D0) * N + st.n;
        // element offset and count of every store below, checked in the debug build
        auto ok = [&](Off o, int n) {
            return LBM_IN(kp, LBM_SITE_PAIR_STORE, a, a + o, n, (size_t)Q * N);
        };
        if (!ODD || i == 0) {
            if (st.active && ok(own, 2)) PairIO<S>::st(a + own, v0[k], v1[k]);
            continue;
        }
        const bool in = !ZWe || st.zo[dz + 1];
        const Off row = (Off)k * N + st.zr[dz + 1] + st.yr[dy + 1];
        if (FAST && dx != 0) {
            const Off e = row + st.x + (Off)dx;
            if (ok(e, 2)) {
                Store<S>::st(a + e, v0[k]);
                Store<S>::st(a + e + 1, v1[k]);
            }
            continue;
        }
        if (st.active && !in && ok(own, 2)) PairIO<S>::st(a + own, v0[k], v1[k]);
        if (dx == 0) {
            if (st.active && in && ok(row + st.x, 2)) PairIO<S>::st(a + row + st.x, v0[k], v1[k]);
        } else if (dx > 0) {
            // element x receives node x - 1, element x + 1 receives node x
            if (st.active && in && !st.left && ok(row + st.x, 2))
                PairIO<S>::st(a + row + st.x, X[k], v0[k]);
            if (st.active && in && st.left && ok(row + st.x + 1, 1))
                Store<S>::st(a + row + st.x + 1, v0[k]);
            // node x + 1 -> x + 2 across the warp edge, or back from an x wall
            const Off o = st.xp2o ? row + st.xp2 : own + 1;
            if (st.active && in && st.right && ok(o, 1)) Store<S>::st(a + o, v1[k]);
        } else {
            // element x receives node x + 1, element x + 1 receives node x + 2
            if (st.active && in && !st.right && ok(row + st.x, 2))
                PairIO<S>::st(a + row + st.x, v1[k], X[k]);
            if (st.active && in && st.right && ok(row + st.x, 1))
                Store<S>::st(a + row + st.x, v1[k]);
            // node x -> x - 1 across the warp edge, or back from an x wall
            const Off o = st.xmo ? row + st.xm : own;
            if (st.active && in && st.left && ok(o, 1)) Store<S>::st(a + o, v0[k]);
        }
    }
}

}  // namespace lbmgpu
