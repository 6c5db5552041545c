// lbm_aux.cu -- initial condition, macroscopic fields, state import/export,
// diagnostics and the small adjoint helpers of the GB300 LBM library.
//
// Diagnostics (Sec. 3.1 and 3.2):
//   chibar(x, z) = (1/ny) sum_y chi,  m(x) = max_z chibar(x, z),
//   x_f = largest x with m(x) >= threshold, moved to the linear crossing
//   between x_f and x_f + 1; front = (x_f + 1/2 - x0) / H;
//   F_w = sum_{x,y} nu (9 u_x(x,y,0) - u_x(x,y,1)) / 3   (Eq. 62-64: the
//   derivative at the wall z = -1/2 of the quadratic through u = 0 there and
//   the first two nodes);
//   budgets sum (rho - 1) and sum chi (= N + sum (chi - 1)).
// Column sums run in FP32 with Kahan compensation, block and grid sums of the
// budgets in FP64, the friction in compensated FP32 pairs; every reduction
// has a fixed order, so results are bitwise reproducible.
#include <type_traits>

#include "lbm_internal.h"

namespace lbmgpu {

template <typename S>
__device__ __forceinline__ constexpr bool is16() { return !std::is_same<S, float>::value; }

// rho - 1, u (with the half-force shift, Eq. 20) and chi - 1 at node n.
template <int Q, int SL, bool ODD, typename S>
__device__ __forceinline__ void node_macros(const KParams& kp, const S* __restrict__ f,
                                            const S* __restrict__ phi, int x, int y, int z,
                                            unsigned n, float& drho, float& ux, float& uy,
                                            float& uz, float& chit) {
    constexpr int NS = ScalarLat<SL>::NS;
    const Stencil st = make_stencil(kp, x, y, z);
    float fv[Q], pv[NS];
    gather<Q, ODD, S, 0, false, true, size_t>(kp, f, st, fv);
    gather<NS, ODD, S, ScalarLat<SL>::D0, rest32<S, SL>(), true, size_t>(kp, phi, st, pv);
    float c = 0.0f;   // chi - 1 (Phi is held as Phi - w, in 16 bits as Phi - chi_s w)
#pragma unroll
    for (int k = 0; k < NS; ++k) c += pv[k];
    if (is16<S>()) c = fmaf(c, kp.isp, kp.chi_s - 1.0f);
    float d = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        d += fv[i];
        jx += cx27(i) * fv[i];
        jy += cy27(i) * fv[i];
        jz += cz27(i) * fv[i];
    }
    if (is16<S>()) { d *= kp.isf; jx *= kp.isf; jy *= kp.isf; jz *= kp.isf; }
    const float irho = 1.0f / (1.0f + d);
    const float chi = 1.0f + c;
    drho = d;
    chit = c;
    ux = (jx + 0.5f * kp.gx * chi) * irho;
    uy = (jy + 0.5f * kp.gy * chi) * irho;
    uz = (jz + 0.5f * kp.gz * chi) * irho;
}

// ---------------------------------------------------------------------------
// Initial condition (Sec. 2.5, Table 1): f = w, Phi_k = w_k chi0, with chi0
// either given or the lock field plus the gate-column perturbation drawn from
// splitmix64(seed ^ n) (Steele, Lea & Flood 2014).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long s) {
    unsigned long long z = s + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

template <int Q, int SL, typename S>
__global__ void init_kernel(KParams kp, S* __restrict__ f, S* __restrict__ phi,
                            const float* __restrict__ chi0, int x0, double amp,
                            unsigned long long seed) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const unsigned n = (unsigned)x + (unsigned)kp.nx * ((unsigned)y + (unsigned)kp.ny * (unsigned)z);
    const size_t N = kp.N;
    float c;  // chi0 - chi_s: the stored deviation of chi (chi0 - 1 in FP32)
    if (chi0) {
        c = chi0[n] - (is16<S>() ? kp.chi_s : 1.0f);
    } else {
        // global column and node index (an x-slab keys the noise by the
        // node's index in the whole box)
        const int xg = x + kp.x_off;
        const unsigned long long ng =
            (unsigned long long)xg +
            (unsigned long long)kp.nxg * ((unsigned long long)y + (unsigned long long)kp.ny * z);
        double v = xg < x0 ? 0.0 : -1.0;
        if (xg == x0 - 1) {
            const double r = (double)(splitmix64(seed ^ ng) >> 11) * 0x1.0p-53;
            v += amp * (2.0 * r - 1.0);
        }
        c = is16<S>() ? (float)(v + (1.0 - (double)kp.chi_s)) : (float)v;
    }
    constexpr int NS = ScalarLat<SL>::NS;
#pragma unroll
    for (int i = 0; i < Q; ++i) store_chk(kp, LBM_SITE_STATE, f, (size_t)i * N + n, Q * N, 0.0f);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const float v = kp.sp * (ScalarLat<SL>::w(k) * c);
        if (rest32<S, SL>() && k == 0) st_chk(kp, LBM_SITE_STATE, rest_row(phi, NS, kp.N), n, N, v);
        else store_chk(kp, LBM_SITE_STATE, phi, (size_t)k * N + n, NS * N, v);
    }
}

__global__ void fill_keys_kernel(unsigned* __restrict__ keys, int n, int* __restrict__ flags,
                                 int reset_flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = 0x007fffffu;  // key of -inf
    if (reset_flags && i == 0) {
        *flags = 0;
        *dbg_record(flags) = DbgRecord{};
    }
}

// ---------------------------------------------------------------------------
template <int Q, int SL, bool ODD, typename S>
__global__ void macros_kernel(KParams kp, const S* __restrict__ f, const S* __restrict__ phi,
                              float* __restrict__ rho, float* __restrict__ u,
                              float* __restrict__ chi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const unsigned n = (unsigned)x + (unsigned)kp.nx * ((unsigned)y + (unsigned)kp.ny * (unsigned)z);
    float d, ux, uy, uz, c;
    node_macros<Q, SL, ODD>(kp, f, phi, x, y, z, n, d, ux, uy, uz, c);
    const size_t N = kp.N;
    if (rho) rho[n] = 1.0f + d;
    if (u) { u[n] = ux; u[N + n] = uy; u[2 * N + n] = uz; }
    if (chi) chi[n] = 1.0f + c;
}

template <int Q, int SL, bool ODD, typename S>
__global__ void get_state_kernel(KParams kp, const S* __restrict__ f, const S* __restrict__ phi,
                                 float* __restrict__ dst) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    constexpr int NS = ScalarLat<SL>::NS;
    const Stencil st = make_stencil(kp, x, y, z);
    const unsigned n = st.n;
    float fv[Q], pv[NS];
    gather<Q, ODD, S, 0, false, true, size_t>(kp, f, st, fv);
    gather<NS, ODD, S, ScalarLat<SL>::D0, rest32<S, SL>(), true, size_t>(kp, phi, st, pv);
    const size_t N = kp.N;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        st_chk(kp, LBM_SITE_STATE, dst, (size_t)i * N + n, (Q + NS) * N,
               is16<S>() ? fv[i] * kp.isf : fv[i]);
#pragma unroll
    for (int k = 0; k < NS; ++k)
        st_chk(kp, LBM_SITE_STATE, dst, (size_t)(Q + k) * N + n, (Q + NS) * N,
               is16<S>() ? phi_canonical(kp, pv[k], ScalarLat<SL>::w(k)) : pv[k]);
}

template <int Q, int SL, typename S>
__global__ void set_state_kernel(KParams kp, S* __restrict__ f, S* __restrict__ phi,
                                 const float* __restrict__ src) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const unsigned n = (unsigned)x + (unsigned)kp.nx * ((unsigned)y + (unsigned)kp.ny * (unsigned)z);
    const size_t N = kp.N;
    constexpr int NS = ScalarLat<SL>::NS;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float v = ld_chk(kp, LBM_SITE_STATE, src, (size_t)i * N + n, (Q + NS) * N);
        store_chk(kp, LBM_SITE_STATE, f, (size_t)i * N + n, Q * N, is16<S>() ? v * kp.sf : v);
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const float v = ld_chk(kp, LBM_SITE_STATE, src, (size_t)(Q + k) * N + n, (Q + NS) * N);
        const float sv = is16<S>() ? phi_stored(kp, v, ScalarLat<SL>::w(k)) : v;
        if (rest32<S, SL>() && k == 0)
            st_chk(kp, LBM_SITE_STATE, rest_row(phi, NS, kp.N), n, N, sv);
        else store_chk(kp, LBM_SITE_STATE, phi, (size_t)k * N + n, NS * N, sv);
    }
}

// ---------------------------------------------------------------------------
// Diagnostics.  One thread per column (x, z), looping over y.
__device__ __forceinline__ unsigned fkey(float v) {
    const unsigned b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
    const unsigned b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}

// (s, c) + (t, d) with an error-free transformation of the leading parts
__device__ __forceinline__ void pair_add(float& s, float& c, float t, float d) {
    float r, e;
    two_sum(s, t, r, e);
    s = r;
    c = c + d + e;
}

constexpr int DIAG_BX = 128;

template <int Q, int SL, bool ODD, typename S>
__global__ void __launch_bounds__(DIAG_BX) diag_columns_kernel(
    KParams kp, const S* __restrict__ f, const S* __restrict__ phi, float* __restrict__ chibar,
    unsigned* __restrict__ colmax, double* __restrict__ part, float* __restrict__ fwpart,
    int* __restrict__ flags) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    double m_rho = 0.0, m_chi = 0.0;
    float fs = 0.0f, fc = 0.0f;
    if (x < kp.nx) {
        Kahan kc, kr, ku;
        int bad = 0;
        for (int y = 0; y < kp.ny; ++y) {
            const unsigned n =
                (unsigned)x + (unsigned)kp.nx * ((unsigned)y + (unsigned)kp.ny * (unsigned)z);
            float d, ux, uy, uz, c;
            node_macros<Q, SL, ODD>(kp, f, phi, x, y, z, n, d, ux, uy, uz, c);
            kc.add(c);
            kr.add(d);
            ku.add(ux);
            if (!(1.0f + d > 0.0f)) bad |= LBM_DEVFLAG_RHO_NONPOS;
            if (!isfinite(d) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz) || !isfinite(c))
                bad |= LBM_DEVFLAG_NONFINITE;
        }
        if (bad) atomicOr(flags, bad);
        const float cb = 1.0f + (kc.s + kc.c) / (float)kp.ny;
        chibar[(size_t)z * kp.nx + x] = cb;
        atomicMax(colmax + x, fkey(cb));
        m_rho = (double)kr.s + (double)kr.c;
        m_chi = (double)kc.s + (double)kc.c;
        if (kp.nz >= 2 && z < 2) {
            const float a = z == 0 ? 3.0f * kp.nu : -kp.nu * (1.0f / 3.0f);
            fs = a * ku.s;
            fc = a * ku.c;
        }
    }
    // block reductions: budgets in FP64, friction in compensated FP32 pairs
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m_rho += __shfl_down_sync(0xffffffffu, m_rho, o);
        m_chi += __shfl_down_sync(0xffffffffu, m_chi, o);
        const float ts = __shfl_down_sync(0xffffffffu, fs, o);
        const float tc = __shfl_down_sync(0xffffffffu, fc, o);
        pair_add(fs, fc, ts, tc);
    }
    __shared__ double sr[DIAG_BX / 32], sc[DIAG_BX / 32];
    __shared__ float ss[DIAG_BX / 32], se[DIAG_BX / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sr[wid] = m_rho; sc[wid] = m_chi; ss[wid] = fs; se[wid] = fc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        float s = 0.0f, c = 0.0f;
        for (int w = 0; w < DIAG_BX / 32; ++w) { a += sr[w]; b += sc[w]; pair_add(s, c, ss[w], se[w]); }
        const unsigned blk = blockIdx.y * gridDim.x + blockIdx.x;
        part[2 * blk] = a;
        part[2 * blk + 1] = b;
        fwpart[2 * blk] = s;
        fwpart[2 * blk + 1] = c;
    }
}

constexpr int FIN_T = 512;

__global__ void __launch_bounds__(FIN_T) diag_finalize_kernel(
    int nx, double nodes, unsigned nblocks, const double* __restrict__ part,
    const float* __restrict__ fwpart, unsigned* __restrict__ colmax, DevDiag* __restrict__ out,
    double thr, int x0, double H, int xlim, int x_off) {
    __shared__ double sa[FIN_T], sb[FIN_T];
    __shared__ float ss[FIN_T], sc[FIN_T];
    __shared__ int sx[FIN_T];
    const int t = threadIdx.x;
    double a = 0.0, b = 0.0;
    float s = 0.0f, c = 0.0f;
    for (unsigned i = t; i < nblocks; i += FIN_T) {
        a += part[2 * i];
        b += part[2 * i + 1];
        pair_add(s, c, fwpart[2 * i], fwpart[2 * i + 1]);
    }
    int xf = -1;
    for (int x = t; x < xlim; x += FIN_T)
        if ((double)fkey_inv(colmax[x]) >= thr) xf = x;
    sa[t] = a; sb[t] = b; ss[t] = s; sc[t] = c; sx[t] = xf;
    __syncthreads();
    for (int w = FIN_T / 2; w > 0; w >>= 1) {
        if (t < w) {
            sa[t] += sa[t + w];
            sb[t] += sb[t + w];
            float s0 = ss[t], c0 = sc[t];
            pair_add(s0, c0, ss[t + w], sc[t + w]);
            ss[t] = s0; sc[t] = c0;
            sx[t] = max(sx[t], sx[t + w]);
        }
        __syncthreads();
    }
    if (t == 0) {
        const int x = sx[0];
        double xn;
        if (x < 0) xn = -1.0;
        else if (x == xlim - 1) xn = (double)x;
        else {
            const double m0 = fkey_inv(colmax[x]), m1 = fkey_inv(colmax[x + 1]);
            xn = x + (m0 - thr) / (m0 - m1);
        }
        if (xn >= 0.0) xn += x_off;   // an x-slab reports its columns in box coordinates
        out->front_node = xn;
        out->front = (xn + 0.5 - x0) / H;
        out->Fw = (double)ss[0] + (double)sc[0];
        out->mass_delta = sa[0];
        out->scalar_mass = nodes + sb[0];   // the columns summed chi - 1
    }
    __syncthreads();
    for (int x = t; x < nx; x += FIN_T) colmax[x] = 0x007fffffu;  // ready for the next call
}

// Adds weight * F_w to *acc.  One thread per (x, y) of the bottom rows.
template <int Q, int SL, bool ODD, typename S>
__global__ void __launch_bounds__(128) fw_kernel(KParams kp, const S* __restrict__ f,
                                                 const S* __restrict__ phi, double* __restrict__ acc,
                                                 double weight) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    double v = 0.0;
    if (x < kp.nx) {
        float d, ux0, ux1, uy, uz, c;
        const unsigned n0 = (unsigned)x + (unsigned)kp.nx * (unsigned)y;
        const unsigned n1 = n0 + kp.nxny;
        node_macros<Q, SL, ODD>(kp, f, phi, x, y, 0, n0, d, ux0, uy, uz, c);
        node_macros<Q, SL, ODD>(kp, f, phi, x, y, 1, n1, d, ux1, uy, uz, c);
        v = (double)(kp.nu * (9.0f * ux0 - ux1) * (1.0f / 3.0f));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double red[4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(acc, weight * (red[0] + red[1] + red[2] + red[3]));
}

__global__ void adjoint_chi0_kernel(unsigned N, int Q, const float* __restrict__ lam,
                                    float* __restrict__ grad) {
    const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float g = 0.0f;
#pragma unroll
    for (int k = 0; k < 7; ++k) g += w7(k) * lam[(size_t)(Q + k) * N + n];
    grad[n] = g;
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
// Front of a canonical FP32 state (Sec. 3.1, reading R11) and its derivative:
// the interpolated front x_f = x + (m0 - thr) / (m0 - m1), m0 = m(x) >= thr >
// m1 = m(x + 1), m(x) = max_z chibar(x, z), depends on the state only through
// chibar at the two maximising (x, z), each the mean over y of chi = 1 +
// sum_k (Phi_k - w_k).  Hence d value / d(Phi_k - w_k) is g0 / ny on the
// column (x, ., z0) and g1 / ny on (x + 1, ., z1), zero elsewhere, with
//   g0 = (thr - m1) / ((m0 - m1)^2 H),  g1 = (m0 - thr) / ((m0 - m1)^2 H).
// When no column reaches thr, or the crossing column is the last one searched
// (front_xlim), the front does not move with the state and the derivative is
// zero.
__global__ void __launch_bounds__(DIAG_BX) front_columns_kernel(KParams kp, int Q, int NS,
                                                                const float* __restrict__ s,
                                                                float* __restrict__ chibar,
                                                                unsigned* __restrict__ colmax) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    if (x >= kp.nx) return;
    Kahan kc;
    for (int y = 0; y < kp.ny; ++y) {
        const unsigned n = (unsigned)x + (unsigned)kp.nx * ((unsigned)y + (unsigned)kp.ny * (unsigned)z);
        float c = 0.0f;
        for (int k = 0; k < NS; ++k) c += s[(size_t)(Q + k) * kp.N + n];
        kc.add(c);
    }
    const float cb = 1.0f + (kc.s + kc.c) / (float)kp.ny;
    chibar[(size_t)z * kp.nx + x] = cb;
    atomicMax(colmax + x, fkey(cb));
}

__global__ void __launch_bounds__(FIN_T) front_finalize_kernel(int nx, int nz,
                                                               const float* __restrict__ chibar,
                                                               unsigned* __restrict__ colmax,
                                                               FrontGrad* __restrict__ out,
                                                               double* __restrict__ value,
                                                               double thr, int x0, double H,
                                                               int xlim) {
    __shared__ int sx[FIN_T];
    const int t = threadIdx.x;
    int xf = -1;
    for (int x = t; x < xlim; x += FIN_T)
        if ((double)fkey_inv(colmax[x]) >= thr) xf = x;
    sx[t] = xf;
    __syncthreads();
    for (int w = FIN_T / 2; w > 0; w >>= 1) {
        if (t < w) sx[t] = max(sx[t], sx[t + w]);
        __syncthreads();
    }
    if (t == 0) {
        const int x = sx[0];
        FrontGrad g;
        g.x = x; g.z0 = 0; g.z1 = 0; g.valid = 0; g.g0 = 0.0; g.g1 = 0.0;
        double xn;
        if (x < 0) xn = -1.0;
        else if (x == xlim - 1) xn = (double)x;
        else {
            const unsigned k0 = colmax[x], k1 = colmax[x + 1];
            const double m0 = fkey_inv(k0), m1 = fkey_inv(k1);
            const double d = m0 - m1;
            xn = x + (m0 - thr) / d;
            g.g0 = (thr - m1) / (d * d * H);
            g.g1 = (m0 - thr) / (d * d * H);
            // the first z attaining each maximum
            int z0 = -1, z1 = -1;
            for (int z = 0; z < nz && (z0 < 0 || z1 < 0); ++z) {
                if (z0 < 0 && fkey(chibar[(size_t)z * nx + x]) == k0) z0 = z;
                if (z1 < 0 && fkey(chibar[(size_t)z * nx + x + 1]) == k1) z1 = z;
            }
            g.z0 = z0; g.z1 = z1;
            g.valid = z0 >= 0 && z1 >= 0;
        }
        g.value = (xn + 0.5 - x0) / H;
        *out = g;
        if (value) *value = g.value;
    }
    __syncthreads();
    for (int x = t; x < nx; x += FIN_T) colmax[x] = 0x007fffffu;  // ready for the next call
}

// lam (zeroed by the caller's launcher) receives the derivative on the 2 ny
// nodes it lives on, in every scalar row.
__global__ void front_scatter_kernel(KParams kp, int Q, int NS, const FrontGrad* __restrict__ g,
                                     float* __restrict__ lam) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= kp.ny || !g->valid) return;
    const float a0 = (float)(g->g0 / kp.ny), a1 = (float)(g->g1 / kp.ny);
    const unsigned n0 = (unsigned)g->x + (unsigned)kp.nx * ((unsigned)y + (unsigned)kp.ny * (unsigned)g->z0);
    const unsigned n1 = (unsigned)(g->x + 1) + (unsigned)kp.nx * ((unsigned)y + (unsigned)kp.ny * (unsigned)g->z1);
    for (int k = 0; k < NS; ++k) {
        lam[(size_t)(Q + k) * kp.N + n0] = a0;
        lam[(size_t)(Q + k) * kp.N + n1] = a1;
    }
}

static inline dim3 node_grid(const KParams& kp) { return dim3((kp.nx + 127) / 128, kp.ny, kp.nz); }

unsigned diag_block_count(int nx, int nz) { return (unsigned)((nx + DIAG_BX - 1) / DIAG_BX) * nz; }

// Calls fn.template operator()<Q, SL, S>() for the model, scalar lattice and
// storage at hand.
template <int Q, int SL, typename Fn>
static cudaError_t dispatch_storage(int storage, Fn&& fn) {
    if (storage == LBM_FP32) return fn.template operator()<Q, SL, float>();
    if (storage == LBM_FP16S) return fn.template operator()<Q, SL, __half>();
    if (storage == LBM_BF16S) return fn.template operator()<Q, SL, __nv_bfloat16>();
    return cudaErrorInvalidValue;
}

template <typename Fn>
static cudaError_t dispatch(Kind k, Fn&& fn) {
    if (k.model == LBM_BGK_SMAG_Q19 && k.scalar == LBM_SCALAR_Q7) return dispatch_storage<19, 7>(k.storage, fn);
    if (k.model == LBM_BGK_SMAG_Q19 && k.scalar == LBM_SCALAR_Q6) return dispatch_storage<19, 6>(k.storage, fn);
    if (k.model == LBM_CUMULANT_Q27 && k.scalar == LBM_SCALAR_Q7) return dispatch_storage<27, 7>(k.storage, fn);
    if (k.model == LBM_CUMULANT_Q27 && k.scalar == LBM_SCALAR_Q27) return dispatch_storage<27, 27>(k.storage, fn);
    return cudaErrorInvalidValue;
}

cudaError_t launch_step(const KParams& kp, Kind k, bool odd, void* f, void* phi, float* save,
                        cudaStream_t st) {
    if (!save && staged_step_applies(kp, k)) return launch_staged_step(kp, k, odd, f, phi, st);
    if (k.model == LBM_BGK_SMAG_Q19) return launch_bgk_step(kp, k.storage, k.scalar, odd, f, phi, save, st);
    if (k.model == LBM_CUMULANT_Q27)
        return launch_cumulant_step(kp, k.storage, k.scalar, odd, f, phi, save, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_init(const KParams& kp, Kind k, const Views& v, const float* chi0, int x0,
                        double amp, uint64_t seed, cudaStream_t st) {
    return dispatch(k, [&]<int Q, int SL, typename S>() {
        init_kernel<Q, SL, S><<<node_grid(kp), 128, 0, st>>>(kp, (S*)v.f, (S*)v.phi, chi0, x0, amp,
                                                              (unsigned long long)seed);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        fill_keys_kernel<<<(kp.nx + 255) / 256, 256, 0, st>>>(v.colmax, kp.nx, v.devflags, 1);
        return cudaGetLastError();
    });
}

cudaError_t launch_macros(const KParams& kp, Kind k, bool odd, const Views& v, float* rho,
                          float* u, float* chi, cudaStream_t st) {
    return dispatch(k, [&]<int Q, int SL, typename S>() {
        if (odd)
            macros_kernel<Q, SL, true, S><<<node_grid(kp), 128, 0, st>>>(kp, (const S*)v.f, (const S*)v.phi, rho, u, chi);
        else
            macros_kernel<Q, SL, false, S><<<node_grid(kp), 128, 0, st>>>(kp, (const S*)v.f, (const S*)v.phi, rho, u, chi);
        return cudaGetLastError();
    });
}

cudaError_t launch_get_state(const KParams& kp, Kind k, bool odd, const Views& v, float* dst,
                             cudaStream_t st) {
    return dispatch(k, [&]<int Q, int SL, typename S>() {
        if (odd)
            get_state_kernel<Q, SL, true, S><<<node_grid(kp), 128, 0, st>>>(kp, (const S*)v.f, (const S*)v.phi, dst);
        else
            get_state_kernel<Q, SL, false, S><<<node_grid(kp), 128, 0, st>>>(kp, (const S*)v.f, (const S*)v.phi, dst);
        return cudaGetLastError();
    });
}

cudaError_t launch_set_state(const KParams& kp, Kind k, const Views& v, const float* src,
                             cudaStream_t st) {
    return dispatch(k, [&]<int Q, int SL, typename S>() {
        set_state_kernel<Q, SL, S><<<node_grid(kp), 128, 0, st>>>(kp, (S*)v.f, (S*)v.phi, src);
        return cudaGetLastError();
    });
}

cudaError_t launch_diag(const KParams& kp, Kind k, bool odd, const Views& v, double threshold,
                        int x0, double H, cudaStream_t st) {
    return dispatch(k, [&]<int Q, int SL, typename S>() {
        dim3 grid((kp.nx + DIAG_BX - 1) / DIAG_BX, kp.nz);
        if (odd)
            diag_columns_kernel<Q, SL, true, S><<<grid, DIAG_BX, 0, st>>>(
                kp, (const S*)v.f, (const S*)v.phi, v.chibar, v.colmax, v.part, v.fwpart, v.devflags);
        else
            diag_columns_kernel<Q, SL, false, S><<<grid, DIAG_BX, 0, st>>>(
                kp, (const S*)v.f, (const S*)v.phi, v.chibar, v.colmax, v.part, v.fwpart, v.devflags);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        diag_finalize_kernel<<<1, FIN_T, 0, st>>>(kp.nx, (double)kp.N, v.diag_blocks, v.part,
                                                  v.fwpart, v.colmax, v.ddiag, threshold, x0, H,
                                                  front_xlim(kp.nx, x0, kp.flags), kp.x_off);
        return cudaGetLastError();
    });
}

// m[x] = max over z of the span-averaged chi of column x (the keys of the
// columns kernel decoded), keys reset for the next diagnostics.
__global__ void column_max_kernel(int nx, unsigned* __restrict__ colmax, float* __restrict__ m) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    m[x] = fkey_inv(colmax[x]);
    colmax[x] = 0x007fffffu;
}

// Front of a whole box from its column maxima m[0 .. nx) (Sec. 3.1, reading
// R11, the search window of front_xlim): out[0] = (x_f + 1/2 - x0) / H,
// out[1] = x_f (-1 when no column reaches the threshold).
__global__ void __launch_bounds__(FIN_T) front_of_columns_kernel(const float* __restrict__ m,
                                                                 int nx, double thr, int x0,
                                                                 double H, int xlim,
                                                                 double* __restrict__ out) {
    __shared__ int sx[FIN_T];
    const int t = threadIdx.x;
    int xf = -1;
    for (int x = t; x < xlim; x += FIN_T)
        if ((double)m[x] >= thr) xf = x;
    sx[t] = xf;
    __syncthreads();
    for (int w = FIN_T / 2; w > 0; w >>= 1) {
        if (t < w) sx[t] = max(sx[t], sx[t + w]);
        __syncthreads();
    }
    if (t == 0) {
        const int x = sx[0];
        double xn;
        if (x < 0) xn = -1.0;
        else if (x == xlim - 1) xn = (double)x;
        else {
            const double m0 = m[x], m1 = m[x + 1];
            xn = x + (m0 - thr) / (m0 - m1);
        }
        out[0] = (xn + 0.5 - x0) / H;
        out[1] = xn;
    }
}

cudaError_t launch_column_max(const KParams& kp, Kind k, bool odd, const Views& v, float* m,
                              cudaStream_t st) {
    cudaError_t e = dispatch(k, [&]<int Q, int SL, typename S>() {
        dim3 grid((kp.nx + DIAG_BX - 1) / DIAG_BX, kp.nz);
        if (odd)
            diag_columns_kernel<Q, SL, true, S><<<grid, DIAG_BX, 0, st>>>(
                kp, (const S*)v.f, (const S*)v.phi, v.chibar, v.colmax, v.part, v.fwpart, v.devflags);
        else
            diag_columns_kernel<Q, SL, false, S><<<grid, DIAG_BX, 0, st>>>(
                kp, (const S*)v.f, (const S*)v.phi, v.chibar, v.colmax, v.part, v.fwpart, v.devflags);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    column_max_kernel<<<(kp.nx + 255) / 256, 256, 0, st>>>(kp.nx, v.colmax, m);
    return cudaGetLastError();
}

cudaError_t launch_front_of_columns(const float* m, int nx, double thr, int x0, double H,
                                    int xlim, double* out, cudaStream_t st) {
    front_of_columns_kernel<<<1, FIN_T, 0, st>>>(m, nx, thr, x0, H, xlim, out);
    return cudaGetLastError();
}

cudaError_t launch_fw_accumulate(const KParams& kp, Kind k, bool odd, const Views& v,
                                 double* acc, double weight, cudaStream_t st) {
    if (kp.nz < 2) return cudaSuccess;
    return dispatch(k, [&]<int Q, int SL, typename S>() {
        dim3 grid((kp.nx + 127) / 128, kp.ny);
        if (odd)
            fw_kernel<Q, SL, true, S><<<grid, 128, 0, st>>>(kp, (const S*)v.f, (const S*)v.phi, acc, weight);
        else
            fw_kernel<Q, SL, false, S><<<grid, 128, 0, st>>>(kp, (const S*)v.f, (const S*)v.phi, acc, weight);
        return cudaGetLastError();
    });
}

cudaError_t launch_front_adjoint(const KParams& kp, int Q, int NS, const Views& v,
                                 const float* state, float* lam, double* value, double threshold,
                                 int x0, double H, cudaStream_t st) {
    dim3 grid((kp.nx + DIAG_BX - 1) / DIAG_BX, kp.nz);
    front_columns_kernel<<<grid, DIAG_BX, 0, st>>>(kp, Q, NS, state, v.chibar, v.colmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    front_finalize_kernel<<<1, FIN_T, 0, st>>>(kp.nx, kp.nz, v.chibar, v.colmax, v.fgrad, value,
                                               threshold, x0, H, front_xlim(kp.nx, x0, kp.flags));
    e = cudaGetLastError();
    if (e != cudaSuccess || !lam) return e;
    e = cudaMemsetAsync(lam, 0, (size_t)(Q + NS) * kp.N * sizeof(float), st);
    if (e != cudaSuccess) return e;
    front_scatter_kernel<<<(kp.ny + 127) / 128, 128, 0, st>>>(kp, Q, NS, v.fgrad, lam);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_chi0(const KParams& kp, int Q, const float* lam0, float* grad,
                                cudaStream_t st) {
    adjoint_chi0_kernel<<<(kp.N + 255) / 256, 256, 0, st>>>(kp.N, Q, lam0, grad);
    return cudaGetLastError();
}

}  // namespace lbmgpu
