// lbm_bgk.cu -- fused AA stream + collide kernel of the D3Q19 BGK-Smagorinsky
// fluid with the D3Q7 scalar and the Boussinesq force, and the hand-written
// discrete adjoint of that step.
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
// The kernel is HBM-bound (about 2 flop per byte): one thread per node, x
// fastest so every population row is read and written as coalesced 128-byte
// segments; no shared memory, no tensor cores.
#include <type_traits>

#include "lbm_aa2.cuh"
#include "lbm_internal.h"

namespace lbmgpu {

// Replaces f (held as f - w) and Phi (held as Phi - w) by their
// post-collision values.  Directions come in opposite pairs (i, i + 1 for odd
// i): with s = f_i + f_opp and d = f_i - f_opp the moments need half the
// additions, and the equilibrium and the Guo source split into a part even
// in c (shared by the pair) and a part odd in c (sign-flipped), which halves
// the per-direction arithmetic.
__device__ __forceinline__ void collide_bgk(const KParams& kp, float (&f)[19], float (&p)[7]) {
    float chit = 0.0f;  // chi - 1
#pragma unroll
    for (int k = 0; k < 7; ++k) chit += p[k];
    const float chi = 1.0f + chit;
    const float Fx = kp.gx * chi, Fy = kp.gy * chi, Fz = kp.gz * chi;

    float drho = f[0], jx = 0.0f, jy = 0.0f, jz = 0.0f;
    float mxx = 0.0f, myy = 0.0f, mzz = 0.0f, mxy = 0.0f, mxz = 0.0f, myz = 0.0f;
#pragma unroll
    for (int i = 1; i < 19; i += 2) {
        const float sp = f[i] + f[i + 1], dm = f[i] - f[i + 1];
        drho += sp;
        if (cx27(i)) { jx += cx27(i) * dm; mxx += sp; }
        if (cy27(i)) { jy += cy27(i) * dm; myy += sp; }
        if (cz27(i)) { jz += cz27(i) * dm; mzz += sp; }
        if (cx27(i) * cy27(i)) mxy += cx27(i) * cy27(i) * sp;
        if (cx27(i) * cz27(i)) mxz += cx27(i) * cz27(i) * sp;
        if (cy27(i) * cz27(i)) myz += cy27(i) * cz27(i) * sp;
    }
    const float rho = 1.0f + drho;
    const float irho = 1.0f / rho;
    const float ux = (jx + 0.5f * Fx) * irho;
    const float uy = (jy + 0.5f * Fy) * irho;
    const float uz = (jz + 0.5f * Fz) * irho;
    const float usq = ux * ux + uy * uy + uz * uz;

    // non-equilibrium second moment (sum c c feq = rho (I/3 + u u), sum c c w = I/3)
    const float d3 = drho * (1.0f / 3.0f);
    const float pxx = mxx - d3 - rho * ux * ux;
    const float pyy = myy - d3 - rho * uy * uy;
    const float pzz = mzz - d3 - rho * uz * uz;
    const float pxy = mxy - rho * ux * uy;
    const float pxz = mxz - rho * ux * uz;
    const float pyz = myz - rho * uy * uz;
    const float q = sqrtf(pxx * pxx + pyy * pyy + pzz * pzz +
                          2.0f * (pxy * pxy + pxz * pxz + pyz * pyz));
    // tau - tau0 without cancellation: X / (2 (s + tau0)), s = sqrt(tau0^2 + X)
    const float X = kp.A * q * irho;
    const float s = sqrtf(kp.tau0 * kp.tau0 + X);
    const float dtau = 0.5f * X / (s + kp.tau0);
    const float om = 1.0f / (kp.tau0 + dtau);
    const float keep = 1.0f - om;
    const float guo = 1.0f - 0.5f * om;
    const float uF = ux * Fx + uy * Fy + uz * Fz;
    // feq_i - w_i = w_i (drho + rho (3 cu + 4.5 cu^2 - 1.5 u.u)),
    // S_i = guo w_i (3 cF - 3 u.F + 9 cu cF)
    const float base = drho - 1.5f * rho * usq;       // even part of (feq - w)/w at cu = 0
    const float gbase = -3.0f * guo * uF;             // even part of S/w at cF = 0
    f[0] = keep * f[0] + w19(0) * (om * base + gbase);
#pragma unroll
    for (int i = 1; i < 19; i += 2) {
        const float cu = cx27(i) * ux + cy27(i) * uy + cz27(i) * uz;
        const float cF = cx27(i) * Fx + cy27(i) * Fy + cz27(i) * Fz;
        const float w = w19(i);
        const float even = w * (om * (base + 4.5f * rho * cu * cu) + gbase + 9.0f * guo * cu * cF);
        const float odd = w * (om * 3.0f * rho * cu + 3.0f * guo * cF);
        f[i] = keep * f[i] + even + odd;
        f[i + 1] = keep * f[i + 1] + even - odd;
    }

    // Phi_eq - w = w (chi - 1 + 4 chi c.u)
    const float omp = 1.0f / (kp.taup0 + kp.kT * dtau);
    const float keepp = 1.0f - omp;
    p[0] = keepp * p[0] + omp * w7(0) * chit;
    const float pe = omp * w7(1) * chit, pa = omp * w7(1) * 4.0f * chi;
    p[1] = keepp * p[1] + pe + pa * ux;
    p[2] = keepp * p[2] + pe - pa * ux;
    p[3] = keepp * p[3] + pe + pa * uy;
    p[4] = keepp * p[4] + pe - pa * uy;
    p[5] = keepp * p[5] + pe + pa * uz;
    p[6] = keepp * p[6] + pe - pa * uz;
}

template <bool ODD, bool SAVE, typename S>
__global__ void __launch_bounds__(128, LBM_STEP_MINB) bgk_step_kernel(KParams kp, S* __restrict__ f,
                                                       S* __restrict__ phi,
                                                       float* __restrict__ save) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const Stencil st = make_stencil(kp, x, blockIdx.y, blockIdx.z);
    const unsigned n = st.n;

    float fv[19], pv[7];
    gather<19, ODD>(kp, f, st, fv);
    gather<7, ODD>(kp, phi, st, pv);
    if (!std::is_same<S, float>::value) {
#pragma unroll
        for (int i = 0; i < 19; ++i) fv[i] *= kp.isf;
#pragma unroll
        for (int k = 0; k < 7; ++k) pv[k] *= kp.isp;
    }
    if (SAVE) {
        const size_t N = kp.N;
#pragma unroll
        for (int i = 0; i < 19; ++i) save[(size_t)i * N + n] = fv[i];
#pragma unroll
        for (int k = 0; k < 7; ++k) save[(size_t)(19 + k) * N + n] = pv[k];
    }
    if (!(kp.flags & LBM_FLAG_NO_COLLIDE)) collide_bgk(kp, fv, pv);
    if (!std::is_same<S, float>::value) {
#pragma unroll
        for (int i = 0; i < 19; ++i) fv[i] *= kp.sf;
#pragma unroll
        for (int k = 0; k < 7; ++k) pv[k] *= kp.sp;
    }
    scatter<19, ODD>(kp, f, st, fv);
    scatter<7, ODD>(kp, phi, st, pv);
}


// Two x-adjacent nodes per thread (nx even): paired population accesses, see
// lbm_aa2.cuh.  Same arithmetic per node as bgk_step_kernel.
template <bool ODD, bool SAVE, typename S>
__global__ void __launch_bounds__(128, LBM_STEP2_MINB) bgk_step2_kernel(KParams kp, S* __restrict__ f,
                                                                    S* __restrict__ phi,
                                                                    float* __restrict__ save) {
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const Stencil2 st = make_stencil2(kp, x, blockIdx.y, blockIdx.z);
    float f0[19], f1[19], p0[7], p1[7];
    gather2<19, ODD>(kp, f, st, f0, f1);
    gather2<7, ODD>(kp, phi, st, p0, p1);
    if (!std::is_same<S, float>::value) {
#pragma unroll
        for (int i = 0; i < 19; ++i) { f0[i] *= kp.isf; f1[i] *= kp.isf; }
#pragma unroll
        for (int k = 0; k < 7; ++k) { p0[k] *= kp.isp; p1[k] *= kp.isp; }
    }
    if (SAVE && st.active) {
        const unsigned N = kp.N;
#pragma unroll
        for (int i = 0; i < 19; ++i)
            *reinterpret_cast<float2*>(save + (size_t)i * N + st.n) = make_float2(f0[i], f1[i]);
#pragma unroll
        for (int k = 0; k < 7; ++k)
            *reinterpret_cast<float2*>(save + (size_t)(19 + k) * N + st.n) = make_float2(p0[k], p1[k]);
    }
    if (!(kp.flags & LBM_FLAG_NO_COLLIDE)) {
        collide_bgk(kp, f0, p0);
        collide_bgk(kp, f1, p1);
    }
    if (!std::is_same<S, float>::value) {
#pragma unroll
        for (int i = 0; i < 19; ++i) { f0[i] *= kp.sf; f1[i] *= kp.sf; }
#pragma unroll
        for (int k = 0; k < 7; ++k) { p0[k] *= kp.sp; p1[k] *= kp.sp; }
    }
    scatter2<19, ODD>(kp, f, st, f0, f1);
    scatter2<7, ODD>(kp, phi, st, p0, p1);
}

template <typename S>
static cudaError_t launch_bgk_typed(const KParams& kp, bool odd, S* f, S* phi, float* save,
                                   cudaStream_t st) {
    if (LBM_BGK_PAIR && kp.nx % 2 == 0) {
        dim3 block(128), grid((kp.nx / 2 + 127) / 128, kp.ny, kp.nz);
        if (save) {
            if (odd) bgk_step2_kernel<true, true, S><<<grid, block, 0, st>>>(kp, f, phi, save);
            else bgk_step2_kernel<false, true, S><<<grid, block, 0, st>>>(kp, f, phi, save);
        } else {
            if (odd) bgk_step2_kernel<true, false, S><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
            else bgk_step2_kernel<false, false, S><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
        }
        return cudaGetLastError();
    }
    dim3 block(128), grid((kp.nx + 127) / 128, kp.ny, kp.nz);
    if (save) {
        if (odd) bgk_step_kernel<true, true, S><<<grid, block, 0, st>>>(kp, f, phi, save);
        else bgk_step_kernel<false, true, S><<<grid, block, 0, st>>>(kp, f, phi, save);
    } else {
        if (odd) bgk_step_kernel<true, false, S><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
        else bgk_step_kernel<false, false, S><<<grid, block, 0, st>>>(kp, f, phi, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_bgk_step(const KParams& kp, int storage, bool odd, void* f, void* phi,
                            float* save, cudaStream_t st) {
    switch (storage) {
        case LBM_FP32: return launch_bgk_typed(kp, odd, (float*)f, (float*)phi, save, st);
        case LBM_FP16S: return launch_bgk_typed(kp, odd, (__half*)f, (__half*)phi, save, st);
        case LBM_BF16S:
            return launch_bgk_typed(kp, odd, (__nv_bfloat16*)f, (__nv_bfloat16*)phi, save, st);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Discrete adjoint of one step.  With T = streaming o collision and the
// objective J = sum_n w_fw(n) F_w(s_n):
//   lam_n = C(s_n)^T P^T lam_{n+1} + w_fw dF_w/ds_n,
// where P^T (transpose of pull streaming with bounce-back) reads the adjoint
// of the post-collision population i at x from lam_{n+1,i}(x + c_i), or from
// lam_{n+1,opp(i)}(x) when x + c_i is beyond a wall, and C^T is the
// reverse-mode derivative of collide_bgk at s_n written out by hand.  The
// kink of q = |Pi| at Pi = 0 takes the subgradient 0.
__global__ void __launch_bounds__(128) bgk_adjoint_kernel(KParams kp, const float* __restrict__ st,
                                                          const float* __restrict__ lamn,
                                                          float* __restrict__ lam,
                                                          double* __restrict__ dcs, float wfw,
                                                          float dAdCs) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const bool active = x < kp.nx;
    const size_t N = kp.N;
    float gcs = 0.0f;
    if (active) {
        const unsigned n =
            (unsigned)x + (unsigned)kp.nx * ((unsigned)y + (unsigned)kp.ny * (unsigned)z);
        // adjoints of the post-collision populations (transpose of the pull:
        // read lam_{n+1} where each post-collision population went)
        const Stencil sn = make_stencil(kp, x, y, z);
        const unsigned N32 = kp.N;
        float mu[19], mup[7];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            bool in = false;
            const unsigned d = i == 0 ? n : nbr(sn, cx27(i), cy27(i), cz27(i), in);
            const unsigned off = (i != 0 && in) ? (unsigned)i * N32 + d : (unsigned)opp(i) * N32 + n;
            mu[i] = lamn ? lamn[off] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            bool in = false;
            const unsigned d = k == 0 ? n : nbr(sn, cx27(k), cy27(k), cz27(k), in);
            const unsigned off = (k != 0 && in) ? (unsigned)(19 + k) * N32 + d
                                                : (unsigned)(19 + opp(k)) * N32 + n;
            mup[k] = lamn ? lamn[off] : 0.0f;
        }
        float f[19], p[7];
#pragma unroll
        for (int i = 0; i < 19; ++i) f[i] = st[(size_t)i * N + n];
#pragma unroll
        for (int k = 0; k < 7; ++k) p[k] = st[(size_t)(19 + k) * N + n];

        // ---- forward recompute (as collide_bgk) ----
        float chit = 0.0f;
#pragma unroll
        for (int k = 0; k < 7; ++k) chit += p[k];
        const float chi = 1.0f + chit;
        const float Fx = kp.gx * chi, Fy = kp.gy * chi, Fz = kp.gz * chi;
        float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
        float mxx = 0.0f, myy = 0.0f, mzz = 0.0f, mxy = 0.0f, mxz = 0.0f, myz = 0.0f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float v = f[i];
            drho += v;
            jx += cx27(i) * v; jy += cy27(i) * v; jz += cz27(i) * v;
            mxx += cx27(i) * cx27(i) * v; myy += cy27(i) * cy27(i) * v; mzz += cz27(i) * cz27(i) * v;
            mxy += cx27(i) * cy27(i) * v; mxz += cx27(i) * cz27(i) * v; myz += cy27(i) * cz27(i) * v;
        }
        const float rho = 1.0f + drho, irho = 1.0f / rho;
        const float ux = (jx + 0.5f * Fx) * irho, uy = (jy + 0.5f * Fy) * irho,
                    uz = (jz + 0.5f * Fz) * irho;
        const float usq = ux * ux + uy * uy + uz * uz;
        const float d3 = drho * (1.0f / 3.0f);
        const float pxx = mxx - d3 - rho * ux * ux, pyy = myy - d3 - rho * uy * uy,
                    pzz = mzz - d3 - rho * uz * uz;
        const float pxy = mxy - rho * ux * uy, pxz = mxz - rho * ux * uz, pyz = myz - rho * uy * uz;
        const float q = sqrtf(pxx * pxx + pyy * pyy + pzz * pzz +
                              2.0f * (pxy * pxy + pxz * pxz + pyz * pyz));
        const float X = kp.A * q * irho;
        const float s = sqrtf(kp.tau0 * kp.tau0 + X);
        const float dtau = 0.5f * X / (s + kp.tau0);
        const float om = 1.0f / (kp.tau0 + dtau);
        const float guo = 1.0f - 0.5f * om;
        const float uF = ux * Fx + uy * Fy + uz * Fz;
        const float omp = 1.0f / (kp.taup0 + kp.kT * dtau);

        // ---- reverse ----
        float gf[19], gp[7];
        float gchi = 0.0f, grho = 0.0f, gux = 0.0f, guy = 0.0f, guz = 0.0f;
        float gFx = 0.0f, gFy = 0.0f, gFz = 0.0f;
        // scalar: Phi* = (1 - omp) Phi + omp Phi_eq
        float gomp = 0.0f;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const float cu = cx27(k) * ux + cy27(k) * uy + cz27(k) * uz;
            const float peq = w7(k) * (chit + 4.0f * chi * cu);
            gp[k] = (1.0f - omp) * mup[k];
            gomp += mup[k] * (peq - p[k]);
            const float gpeq = omp * mup[k];
            gchi += gpeq * w7(k) * (1.0f + 4.0f * cu);
            const float a = gpeq * w7(k) * chi * 4.0f;
            gux += a * cx27(k); guy += a * cy27(k); guz += a * cz27(k);
        }
        // tau_Phi = taup0 + kT dtau
        float gtau = -gomp * omp * omp * kp.kT;
        // fluid: f* = (1 - om) f + om feq + (1 - om/2) B
        float gom = 0.0f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float cxi = cx27(i), cyi = cy27(i), czi = cz27(i);
            const float cu = cxi * ux + cyi * uy + czi * uz;
            const float cF = cxi * Fx + cyi * Fy + czi * Fz;
            const float w = w19(i);
            const float pol = 3.0f * cu + 4.5f * cu * cu - 1.5f * usq;
            const float feq = w * (drho + rho * pol);
            const float B = w * (3.0f * cF - 3.0f * uF + 9.0f * cu * cF);
            gf[i] = (1.0f - om) * mu[i];
            gom += mu[i] * (feq - f[i]) - 0.5f * mu[i] * B;
            const float gfeq = om * mu[i];
            const float gB = guo * mu[i];
            grho += gfeq * w * (1.0f + pol);
            const float a = gfeq * w * rho;   // d feq / du = w rho (3 c + 9 cu c - 3 u)
            gux += a * (3.0f * cxi + 9.0f * cu * cxi - 3.0f * ux);
            guy += a * (3.0f * cyi + 9.0f * cu * cyi - 3.0f * uy);
            guz += a * (3.0f * czi + 9.0f * cu * czi - 3.0f * uz);
            const float b = gB * w;           // dB/dF = w (3 c - 3 u + 9 cu c), dB/du = w (-3 F + 9 cF c)
            gFx += b * (3.0f * cxi - 3.0f * ux + 9.0f * cu * cxi);
            gFy += b * (3.0f * cyi - 3.0f * uy + 9.0f * cu * cyi);
            gFz += b * (3.0f * czi - 3.0f * uz + 9.0f * cu * czi);
            gux += b * (-3.0f * Fx + 9.0f * cF * cxi);
            guy += b * (-3.0f * Fy + 9.0f * cF * cyi);
            guz += b * (-3.0f * Fz + 9.0f * cF * czi);
        }
        gtau += -gom * om * om;
        // dtau = (s - tau0)/2, s = sqrt(tau0^2 + X): d dtau / dX = 1 / (4 s)
        const float gX = gtau / (4.0f * s);
        // X = A q / rho
        const float gq = gX * kp.A * irho;
        grho += -gX * X * irho;
        gcs = gX * q * irho * dAdCs;
        // q = |Pi| (subgradient 0 at Pi = 0); independent entries xx, yy, zz, xy, xz, yz
        float gpxx = 0.0f, gpyy = 0.0f, gpzz = 0.0f, gpxy = 0.0f, gpxz = 0.0f, gpyz = 0.0f;
        if (q > 0.0f) {
            const float r = gq / q;
            gpxx = r * pxx; gpyy = r * pyy; gpzz = r * pzz;
            gpxy = 2.0f * r * pxy; gpxz = 2.0f * r * pxz; gpyz = 2.0f * r * pyz;
        }
        // Pi_ab = M_ab - (drho / 3) delta_ab - rho u_a u_b
        grho += -(gpxx + gpyy + gpzz) * (1.0f / 3.0f) -
                (gpxx * ux * ux + gpyy * uy * uy + gpzz * uz * uz + gpxy * ux * uy +
                 gpxz * ux * uz + gpyz * uy * uz);
        gux += -rho * (2.0f * gpxx * ux + gpxy * uy + gpxz * uz);
        guy += -rho * (2.0f * gpyy * uy + gpxy * ux + gpyz * uz);
        guz += -rho * (2.0f * gpzz * uz + gpxz * ux + gpyz * uy);
        // objective: F_w = sum_{x,y} nu (9 u_x(z=0) - u_x(z=1)) / 3   (Eq. 62-64)
        if (wfw != 0.0f && kp.nz >= 2) {
            if (z == 0) gux += wfw * 3.0f * kp.nu;
            else if (z == 1) gux += -wfw * kp.nu * (1.0f / 3.0f);
        }
        // u = (j + F/2) / rho
        const float gjx = gux * irho, gjy = guy * irho, gjz = guz * irho;
        gFx += 0.5f * gux * irho; gFy += 0.5f * guy * irho; gFz += 0.5f * guz * irho;
        grho += -(gux * ux + guy * uy + guz * uz) * irho;
        // j = sum c f, rho = 1 + sum f, M = sum c c f
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float cxi = cx27(i), cyi = cy27(i), czi = cz27(i);
            gf[i] += grho + cxi * gjx + cyi * gjy + czi * gjz + gpxx * cxi * cxi +
                     gpyy * cyi * cyi + gpzz * czi * czi + gpxy * cxi * cyi + gpxz * cxi * czi +
                     gpyz * cyi * czi;
        }
        // F = g' chi e^g, chi = 1 + sum (Phi - w)
        gchi += gFx * kp.gx + gFy * kp.gy + gFz * kp.gz;
#pragma unroll
        for (int k = 0; k < 7; ++k) gp[k] += gchi;
#pragma unroll
        for (int i = 0; i < 19; ++i) lam[(size_t)i * N + n] = gf[i];
#pragma unroll
        for (int k = 0; k < 7; ++k) lam[(size_t)(19 + k) * N + n] = gp[k];
    }
    // dJ/dC_s: block reduction in FP64, one atomic per block
    if (dcs) {
        double v = (double)gcs;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __shared__ double red[4];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            if (t != 0.0) atomicAdd(dcs, t);
        }
    }
}

cudaError_t launch_adjoint_step(const KParams& kp, const float* state, const float* lam_next,
                                float* lam, double* dcs, float wfw, float dAdCs, cudaStream_t st) {
    dim3 block(128), grid((kp.nx + 127) / 128, kp.ny, kp.nz);
    bgk_adjoint_kernel<<<grid, block, 0, st>>>(kp, state, lam_next, lam, dcs, wfw, dAdCs);
    return cudaGetLastError();
}

}  // namespace lbmgpu
