// lbm_common.cuh -- device-side building blocks shared by the kernels of the
// GB300 lock-exchange LBM library: lattice constants, kernel parameters,
// storage conversions and the AA-pattern gather / scatter.
//
// Lattices (Sec. 2.3.1): D3Q19 in the order of Eq. 23 with the weights of
// Eq. 24; D3Q27 = D3Q19 followed by the eight corners in opposite pairs;
// D3Q7 for the scalar (rest, +-x, +-y, +-z; weights 1/4 and 1/8, c_s^2 = 1/4).
// In every set the direction opposite to i >= 1 is i + 1 for odd i and i - 1
// for even i.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/lbm.h"

namespace lbmgpu {

// ---------------------------------------------------------------------------
// Lattice constants (compile-time; folded after loop unrolling).

__host__ __device__ constexpr int cx27(int i) {
    constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0,
                           1, -1, 1, -1, 1, -1, -1, 1};
    return t[i];
}
__host__ __device__ constexpr int cy27(int i) {
    constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1,
                           1, -1, 1, -1, -1, 1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int cz27(int i) {
    constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1,
                           1, -1, -1, 1, 1, -1, 1, -1};
    return t[i];
}
// D3Q19 is the first 19 entries of the D3Q27 order.
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

__host__ __device__ constexpr float w19(int i) {
    return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr float w27(int i) {
    return i == 0 ? 8.0f / 27.0f : (i <= 6 ? 2.0f / 27.0f : (i <= 18 ? 1.0f / 54.0f : 1.0f / 216.0f));
}
template <int Q>
__host__ __device__ constexpr float wq(int i) { return Q == 19 ? w19(i) : w27(i); }

// D3Q7: first 7 entries of the same order.
__host__ __device__ constexpr float w7(int k) { return k == 0 ? 0.25f : 0.125f; }

// Scalar lattices (the value of lbm_params.scalar in brackets):
//   D3Q7  [0] BGK, c_s^2 = 1/4 (directions 0..6);
//   D3Q6  [1] BGK, c_s^2 = 1/3, w = 1/6, no rest population (directions 1..6,
//             the order of Eq. 31);
//   D3Q27 [2] factorized central moments (directions 0..26).
// Population k of a lattice is direction k + D0 of the D3Q27 order.
template <int SL> struct ScalarLat;
template <> struct ScalarLat<7> {
    static constexpr int NS = 7, D0 = 0;
    static __host__ __device__ constexpr float w(int k) { return w7(k); }
};
template <> struct ScalarLat<6> {
    static constexpr int NS = 6, D0 = 1;
    static __host__ __device__ constexpr float w(int) { return 1.0f / 6.0f; }
};
template <> struct ScalarLat<27> {
    static constexpr int NS = 27, D0 = 0;
    static __host__ __device__ constexpr float w(int k) { return w27(k); }
};

// ---------------------------------------------------------------------------
// Kernel parameters, derived once on the host from lbm_params.
struct KParams {
    int nx, ny, nz, flags;
    unsigned N;          // nodes
    unsigned nxny;
    float tau0;          // 3 nu + 1/2                          (Eq. 25)
    float A;             // 18 sqrt(2) C_s^2                    (Eq. 34, reading R3)
    float taup0;         // 1/2 + 4 D                           (Eq. 30 on D3Q7)
    float kT;            // 4 / (3 Sc_T): tau_Phi = taup0 + kT (tau - tau0) (Eq. 35)
    float om1, om2;      // cumulant shear and bulk rates       (Eq. 58)
    float omD;           // D3Q27 scalar: first-order rate from D (Eq. 51)
    float gx, gy, gz;    // g' e^g                               (Eq. 11)
    float sf, isf;       // storage scale of f - w and its inverse
    float sp, isp;       // storage scale of Phi and its inverse
    float nu;            // molecular viscosity (wall friction, Eq. 62)
    float omp0;          // 1 / taup0: the scalar rate of the cumulant model (molecular D)
    int* devflags;       // sticky device flags (LBM_DEVFLAG_*) of the context
    int x_off, nxg;      // x-slab: global x of local column 0, nx of the whole box
    int wide;            // (Q + NS) N >= 2^32: 64-bit element offsets in the step kernels
    float chi_s;         // the scalar is stored as sp (Phi - chi_s w): 1 in FP32 storage
};

// ---------------------------------------------------------------------------
// Index checks of the debug build (compiled with LBM_DEBUG).  Before each
// population access of the step, halo, adjoint and state-transfer kernels,
// LBM_IN(kp, site, base, p, n, extent) checks that the n elements at p lie in
// the array [base, base + extent) (element counts).  A failed check counts
// itself in the context's DbgRecord (after its two device flag words),
// records the first failure, sets LBM_DEVFLAG_BOUNDS and yields false: the
// caller skips the access, and a skipped load gives 0.  With the test hook
// LBM_FLAG_TEST_BOUNDS every check takes half the true extent, so accesses to
// the upper half of each array fail the check while no access ever leaves
// its array.  Without LBM_DEBUG, LBM_IN is the constant true and evaluates
// nothing.
struct DbgRecord {
    unsigned long long count;   // failed checks
    long long off, extent;      // first failure: element offset and the extent checked
    int site, pad;              // first failure: LBM_SITE_*
};

__host__ __device__ inline DbgRecord* dbg_record(int* devflags) {
    return reinterpret_cast<DbgRecord*>(devflags + 2);
}

#ifdef LBM_DEBUG
static __device__ __noinline__ void dbg_fail(int* devflags, int site, long long off,
                                             long long extent) {
    if (!devflags) return;
    DbgRecord* r = dbg_record(devflags);
    if (atomicAdd(&r->count, 1ull) == 0ull) {
        r->site = site;
        r->off = off;
        r->extent = extent;
    }
    atomicOr(devflags, LBM_DEVFLAG_BOUNDS);
}

template <typename T>
__device__ __forceinline__ bool dbg_in(int* devflags, int flags, int site, const T* base,
                                       const T* p, long long n, long long extent) {
    if (flags & LBM_FLAG_TEST_BOUNDS) extent /= 2;
    const long long off = (long long)(p - base);
    if (off >= 0 && off + n <= extent) return true;
    dbg_fail(devflags, site, off, extent);
    return false;
}
#define LBM_IN(kp, site, base, p, n, extent) \
    (::lbmgpu::dbg_in((kp).devflags, (kp).flags, (site), (base), (p), (long long)(n), \
                      (long long)(extent)))
#else
#define LBM_IN(kp, site, base, p, n, extent) true
#endif

// ---------------------------------------------------------------------------
// Tuning of the step kernels (compile-time): minimum resident blocks per SM
// requested from the register allocator, and whether population traffic uses
// the streaming (evict-first) cache policy.  Each population is touched once
// per step, so nothing is lost by not keeping it cached.
#ifndef LBM_STEP_MINB
#define LBM_STEP_MINB 4
#endif
#ifndef LBM_STREAMING_HINTS
#define LBM_STREAMING_HINTS 0
#endif
// Two nodes per thread with paired accesses when nx is even (lbm_aa2.cuh):
// measured faster for the BGK model (all storages); the cumulant model, whose
// collision needs more registers per node, keeps one node per thread.
#ifndef LBM_BGK_PAIR
#define LBM_BGK_PAIR 1
#endif
#ifndef LBM_STEP2_MINB
#define LBM_STEP2_MINB 4
#endif

// ---------------------------------------------------------------------------
// Storage types: FP32, or FP16 / BF16 with round-to-nearest-even.
template <typename T>
__device__ __forceinline__ T ld_pop(const T* p) {
#if LBM_STREAMING_HINTS
    return __ldcs(p);
#else
    return *p;
#endif
}
template <typename T>
__device__ __forceinline__ void st_pop(T* p, T v) {
#if LBM_STREAMING_HINTS
    __stcs(p, v);
#else
    *p = v;
#endif
}

template <typename S> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float* p) { return ld_pop(p); }
    static __device__ __forceinline__ void st(float* p, float v) { st_pop(p, v); }
    static __device__ __forceinline__ float rnd(float v) { return v; }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(ld_pop(p)); }
    static __device__ __forceinline__ void st(__half* p, float v) { st_pop(p, __float2half_rn(v)); }
    static __device__ __forceinline__ float rnd(float v) { return __half2float(__float2half_rn(v)); }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) {
        return __bfloat162float(ld_pop(p));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) {
        st_pop(p, __float2bfloat16_rn(v));
    }
    static __device__ __forceinline__ float rnd(float v) {
        return __bfloat162float(__float2bfloat16_rn(v));
    }
};

// ---------------------------------------------------------------------------
// With 16-bit storage the scalar's rest population is kept in FP32: a row of
// N floats after the NS 16-bit rows of the scalar array, at the next 256-byte
// boundary (the 16-bit row of the rest population is unused).  Each step the
// storage roundings of the moving populations are added to it (feed_rest),
// so the 16-bit forms conserve sum chi up to FP32 rounding: rounding the
// scalar to 16 bits otherwise loses or gains mass systematically wherever a
// node's increments fall below half an ulp (the tails of the interface).
__host__ __device__ constexpr size_t rest_row_bytes(int rows, size_t N, size_t es) {
    return (rows * N * es + 255) / 256 * 256;
}
template <typename S>
__device__ __forceinline__ float* rest_row(S* a, int rows, unsigned N) {
    return reinterpret_cast<float*>(reinterpret_cast<char*>(a) + rest_row_bytes(rows, N, sizeof(S)));
}
template <typename S>
__device__ __forceinline__ const float* rest_row(const S* a, int rows, unsigned N) {
    return reinterpret_cast<const float*>(reinterpret_cast<const char*>(a) +
                                          rest_row_bytes(rows, N, sizeof(S)));
}
template <typename S, int SL>
__host__ __device__ constexpr bool rest32() {
    return !std::is_same<S, float>::value && SL != 6;
}

// Rounds populations 1 .. NS-1 (storage units) to the storage type and adds
// their rounding errors to population 0, which is stored in FP32.
template <typename S, int NS>
__device__ __forceinline__ void feed_rest(float (&p)[NS]) {
    float e = 0.0f;
#pragma unroll
    for (int k = 1; k < NS; ++k) {
        const float r = Store<S>::rnd(p[k]);
        e += p[k] - r;
        p[k] = r;
    }
    p[0] += e;
}

// ---------------------------------------------------------------------------
// Neighbourhood of one node, computed once per thread: the node indices of
// the rows (y + dy, z + dz) and the columns x + dx, with y always periodic
// and x, z bounded by half-way bounce-back walls unless the periodic flags
// are set.  Node indices are 32-bit (N < 2^31); element offsets row * N + n
// are computed in the type Off of the gather / scatter: 32-bit in the step
// kernels where (Q + NS) N < 2^32 (KParams::wide false), 64-bit otherwise and
// in the auxiliary kernels.
struct Stencil {
    unsigned n;        // this node
    unsigned zr[3];    // (z + dz) * nx * ny for dz = -1, 0, 1
    unsigned yr[3];    // (y + dy) * nx       for dy = -1, 0, 1
    unsigned xc[3];    // x + dx              for dx = -1, 0, 1
    bool zo[3], xo[3]; // neighbour in the fluid (or wrapped)
};

__device__ __forceinline__ Stencil make_stencil(const KParams& kp, int x, int y, int z) {
    Stencil s;
    const bool px = (kp.flags & LBM_FLAG_PERIODIC_X) != 0;
    const bool pz = (kp.flags & LBM_FLAG_PERIODIC_Z) != 0;
    const int ym = y == 0 ? kp.ny - 1 : y - 1, yp = y == kp.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? kp.nz - 1 : z - 1, zp = z == kp.nz - 1 ? 0 : z + 1;
    const int xm = x == 0 ? kp.nx - 1 : x - 1, xp = x == kp.nx - 1 ? 0 : x + 1;
    s.yr[0] = (unsigned)ym * kp.nx; s.yr[1] = (unsigned)y * kp.nx; s.yr[2] = (unsigned)yp * kp.nx;
    s.zr[0] = (unsigned)zm * kp.nxny; s.zr[1] = (unsigned)z * kp.nxny; s.zr[2] = (unsigned)zp * kp.nxny;
    s.xc[0] = (unsigned)xm; s.xc[1] = (unsigned)x; s.xc[2] = (unsigned)xp;
    s.zo[0] = z > 0 || pz; s.zo[1] = true; s.zo[2] = z < kp.nz - 1 || pz;
    s.xo[0] = x > 0 || px; s.xo[1] = true; s.xo[2] = x < kp.nx - 1 || px;
    s.n = s.zr[1] + s.yr[1] + s.xc[1];
    return s;
}

// Node index of the neighbour displaced by (dx, dy, dz); `inside` is false
// when it lies beyond a wall.
__device__ __forceinline__ unsigned nbr(const Stencil& s, int dx, int dy, int dz, bool& inside) {
    inside = s.xo[dx + 1] && s.zo[dz + 1];
    return s.zr[dz + 1] + s.yr[dy + 1] + s.xc[dx + 1];
}

// ---------------------------------------------------------------------------
// AA pattern, in place on one array per population set (Q fluid, 7 scalar).
//
// Slot i of node n after an even number of steps holds f_i(n), the streamed
// pre-collision value.  Even steps read slot i of node n and write f*_i to
// slot opp(i) of node n.  Odd steps read f_i(n) = f*_i(n - c_i) from slot
// opp(i) of node n - c_i and write f*_i to slot i of node n + c_i.  At a wall
// the bounce-back partner is the node itself: an odd-step read of a
// population whose upwind node is a wall takes slot i of node n (where the
// even step put f*_opp(i)), and an odd-step write towards a wall goes to slot
// opp(i) of node n.  Each location is read and then written by exactly one
// thread in each step, so the update is race-free in place.

// Population k is direction dk = k + D0 and lives in row k; its opposite
// direction's row is opp(dk) - D0.
// R32: population 0 (direction 0) lives in the FP32 rest row (rest_row).
// W: the node may have a wall neighbour; false when every neighbour is known
// to be in the fluid (the wall selects are then skipped).
// One population k (of Q): the read of the gather, the write of the scatter.
template <int Q, bool ODD, typename S, int D0 = 0, bool R32 = false, bool W = true,
          typename Off = unsigned>
__device__ __forceinline__ float gather_one(const KParams& kp, const S* __restrict__ a,
                                            const Stencil& st, int k) {
    const unsigned N = kp.N;
    const int d = k + D0;
    if (R32 && d == 0) {
        const float* r = rest_row(a, Q, N);
        return LBM_IN(kp, LBM_SITE_GATHER, r, r + st.n, 1, N) ? ld_pop(r + st.n) : 0.0f;
    }
    Off off = (Off)k * N + st.n;
    if (ODD && d != 0) {
        bool in;
        const unsigned s = nbr(st, -cx27(d), -cy27(d), -cz27(d), in);
        off = (!W || in) ? (Off)(opp(d) - D0) * N + s : off;
    }
    return LBM_IN(kp, LBM_SITE_GATHER, a, a + off, 1, (size_t)Q * N) ? Store<S>::ld(a + off)
                                                                      : 0.0f;
}

template <int Q, bool ODD, typename S, int D0 = 0, bool R32 = false, bool W = true,
          typename Off = unsigned>
__device__ __forceinline__ void scatter_one(const KParams& kp, S* __restrict__ a,
                                            const Stencil& st, int k, float v) {
    const unsigned N = kp.N;
    const int d = k + D0;
    if (R32 && d == 0) {
        float* r = rest_row(a, Q, N);
        if (LBM_IN(kp, LBM_SITE_SCATTER, r, r + st.n, 1, N)) st_pop(r + st.n, v);
        return;
    }
    Off off = (Off)(opp(d) - D0) * N + st.n;
    if (ODD && d != 0) {
        bool in;
        const unsigned t = nbr(st, cx27(d), cy27(d), cz27(d), in);
        off = (!W || in) ? (Off)k * N + t : off;
    }
    if (LBM_IN(kp, LBM_SITE_SCATTER, a, a + off, 1, (size_t)Q * N)) Store<S>::st(a + off, v);
}

template <int Q, bool ODD, typename S, int D0 = 0, bool R32 = false, bool W = true,
          typename Off = unsigned>
__device__ __forceinline__ void gather(const KParams& kp, const S* __restrict__ a,
                                       const Stencil& st, float (&v)[Q]) {
#pragma unroll
    for (int k = 0; k < Q; ++k) v[k] = gather_one<Q, ODD, S, D0, R32, W, Off>(kp, a, st, k);
}

template <int Q, bool ODD, typename S, int D0 = 0, bool R32 = false, bool W = true,
          typename Off = unsigned>
__device__ __forceinline__ void scatter(const KParams& kp, S* __restrict__ a, const Stencil& st,
                                        const float (&v)[Q]) {
#pragma unroll
    for (int k = 0; k < Q; ++k) scatter_one<Q, ODD, S, D0, R32, W, Off>(kp, a, st, k, v[k]);
}

// Element o of an FP32 buffer of `extent` elements (adjoint fields, saved
// states), loaded or stored under the debug build's index check.
__device__ __forceinline__ float ld_chk(const KParams& kp, int site, const float* __restrict__ a,
                                        size_t o, size_t extent) {
    return LBM_IN(kp, site, a, a + o, 1, extent) ? a[o] : 0.0f;
}
__device__ __forceinline__ void st_chk(const KParams& kp, int site, float* __restrict__ a,
                                       size_t o, size_t extent, float v) {
    if (LBM_IN(kp, site, a, a + o, 1, extent)) a[o] = v;
}

template <typename S>
__device__ __forceinline__ void store_chk(const KParams& kp, int site, S* __restrict__ a, size_t o,
                                          size_t extent, float v) {
    if (LBM_IN(kp, site, a, a + o, 1, extent)) Store<S>::st(a + o, v);
}

// With 16-bit storage the scalar populations are held as scale_phi (Phi_k -
// chi_s w_k), deviations from the scalar field chi_s (KParams::chi_s); the
// FP32 form of the state (lbm_get_state, saved steps) is Phi_k - w_k.  The
// collisions see chi = chi_s + sum_k (stored_k) / scale_phi, and their
// equilibria keep the same form in the stored units.  These convert one
// population of weight w.
__device__ __forceinline__ float phi_canonical(const KParams& kp, float v, float w) {
    return fmaf(v, kp.isp, w * (kp.chi_s - 1.0f));
}
__device__ __forceinline__ float phi_stored(const KParams& kp, float c, float w) {
    return (c - w * (kp.chi_s - 1.0f)) * kp.sp;
}

// Saved pre-collision state (lbm_step_save): row r of node n in a buffer of
// `rows` FP32 rows of N values.
__device__ __forceinline__ void save_pop(const KParams& kp, float* __restrict__ save, int rows,
                                         int r, unsigned n, float v) {
    const size_t o = (size_t)r * kp.N + n;
    if (LBM_IN(kp, LBM_SITE_STATE, save, save + o, 1, (size_t)rows * kp.N)) save[o] = v;
}

// Columns searched for the front (Sec. 3.1 with reading R11): all of them
// with walls at the x ends; with periodic ends (Fig. 4b: a periodic array of
// currents) the half of the ring ahead of the lock, x < (nx + x0) / 2, so that
// the current leaving the lock to the left and re-entering at x = nx - 1 is
// not taken for the front.
__host__ __device__ inline int front_xlim(int nx, int x0, int flags) {
    if (!(flags & LBM_FLAG_PERIODIC_X)) return nx;
    const int h = (nx + x0) / 2;
    return h < 1 ? 1 : h;
}

// True when no node of this block of blockDim.x x-consecutive nodes has a
// wall neighbour (uniform over the block).
__device__ __forceinline__ bool block_interior(const KParams& kp) {
    const int x0 = blockIdx.x * blockDim.x, z = blockIdx.z;
    const bool ix = (kp.flags & LBM_FLAG_PERIODIC_X) || (x0 >= 1 && x0 + (int)blockDim.x <= kp.nx - 1);
    const bool iz = (kp.flags & LBM_FLAG_PERIODIC_Z) || (z >= 1 && z <= kp.nz - 2);
    return ix && iz;
}

// Legacy form used by the auxiliary kernels: neighbour of (x, y, z) displaced
// by (dx, dy, dz), false beyond a wall.
__device__ __forceinline__ bool neighbour(const KParams& kp, int x, int y, int z, int dx, int dy,
                                          int dz, unsigned& idx) {
    int xn = x + dx, yn = y + dy, zn = z + dz;
    if (yn < 0) yn += kp.ny;
    else if (yn >= kp.ny) yn -= kp.ny;
    if (xn < 0 || xn >= kp.nx) {
        if (!(kp.flags & LBM_FLAG_PERIODIC_X)) return false;
        xn = xn < 0 ? xn + kp.nx : xn - kp.nx;
    }
    if (zn < 0 || zn >= kp.nz) {
        if (!(kp.flags & LBM_FLAG_PERIODIC_Z)) return false;
        zn = zn < 0 ? zn + kp.nz : zn - kp.nz;
    }
    idx = (unsigned)xn + (unsigned)kp.nx * ((unsigned)yn + (unsigned)kp.ny * (unsigned)zn);
    return true;
}

// ---------------------------------------------------------------------------
// Reciprocal, quotient and square root inside the collisions: IEEE-rounded
// on the FP32 path, the hardware approximations (relative error about 1e-7)
// where the results are rounded to 16-bit storage (2^-11 or 2^-8) anyway.
template <bool APPROX>
__device__ __forceinline__ float crcp(float x) { return APPROX ? __fdividef(1.0f, x) : 1.0f / x; }
template <bool APPROX>
__device__ __forceinline__ float cdiv(float a, float b) { return APPROX ? __fdividef(a, b) : a / b; }
template <bool APPROX>
__device__ __forceinline__ float csqrt(float x) {
    return APPROX ? (x > 0.0f ? x * rsqrtf(x) : 0.0f) : sqrtf(x);
}

// ---------------------------------------------------------------------------
// Error-free transformation used by the compensated FP32 sums.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v) {
        float t, e;
        two_sum(s, v, t, e);
        s = t;
        c = __fadd_rn(c, e);
    }
};

}  // namespace lbmgpu
