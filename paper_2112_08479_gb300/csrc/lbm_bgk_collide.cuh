// lbm_bgk_collide.cuh -- the per-node collision of the D3Q19 BGK-Smagorinsky
// fluid with the D3Q7 scalar and the Boussinesq force, shared by the AA step
// kernels, the out-of-place recompute and the adjoint.
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
#pragma once

#include "lbm_common.cuh"

namespace lbmgpu {

// Replaces f (held as f - w) and Phi (held as Phi - w) by their
// post-collision values.  Directions come in opposite pairs (i, i + 1 for odd
// i): with s = f_i + f_opp and d = f_i - f_opp the moments need half the
// additions, and the equilibrium and the Guo source split into a part even
// in c (shared by the pair) and a part odd in c (sign-flipped), which halves
// the per-direction arithmetic.
//
// SCALED: f and p hold the 16-bit storage units scale_f (f - w) and
// scale_phi (Phi - w); the scales are applied to the few moments and output
// terms instead of to every population, and the divisions and square roots
// use the hardware approximations (crcp, cdiv, csqrt).
//
// SL: scalar lattice, D3Q7 (c_s^2 = 1/4) or D3Q6 (Eq. 29-31 as printed,
// c_s^2 = 1/3, w = 1/6, no rest population).
template <bool SCALED = false, int SL = 7>
__device__ __forceinline__ void collide_bgk(const KParams& kp, float (&f)[19],
                                            float (&p)[ScalarLat<SL>::NS]) {
    static_assert(SL == 7 || SL == 6, "BGK runs with the D3Q7 or D3Q6 scalar");
    constexpr int NS = ScalarLat<SL>::NS;
    const float isf = SCALED ? kp.isf : 1.0f, isp = SCALED ? kp.isp : 1.0f;
    const float sf = SCALED ? kp.sf : 1.0f, sp = SCALED ? kp.sp : 1.0f;
    float chs = 0.0f;  // scale_phi (chi - 1)
#pragma unroll
    for (int k = 0; k < NS; ++k) chs += p[k];
    const float chit = chs * isp;  // chi - chi_s
    const float chi = kp.chi_s + chit;
    const float Fx = kp.gx * chi, Fy = kp.gy * chi, Fz = kp.gz * chi;

    float drho = f[0], jx = 0.0f, jy = 0.0f, jz = 0.0f;
    float mxx = 0.0f, myy = 0.0f, mzz = 0.0f, mxy = 0.0f, mxz = 0.0f, myz = 0.0f;
#pragma unroll
    for (int i = 1; i < 19; i += 2) {
        const float sm = f[i] + f[i + 1], dm = f[i] - f[i + 1];
        drho += sm;
        if (cx27(i)) { jx += cx27(i) * dm; mxx += sm; }
        if (cy27(i)) { jy += cy27(i) * dm; myy += sm; }
        if (cz27(i)) { jz += cz27(i) * dm; mzz += sm; }
        if (cx27(i) * cy27(i)) mxy += cx27(i) * cy27(i) * sm;
        if (cx27(i) * cz27(i)) mxz += cx27(i) * cz27(i) * sm;
        if (cy27(i) * cz27(i)) myz += cy27(i) * cz27(i) * sm;
    }
    if (SCALED) {
        drho *= isf; jx *= isf; jy *= isf; jz *= isf;
        mxx *= isf; myy *= isf; mzz *= isf; mxy *= isf; mxz *= isf; myz *= isf;
    }
    const float rho = 1.0f + drho;
    const float irho = crcp<SCALED>(rho);
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
    const float q = csqrt<SCALED>(pxx * pxx + pyy * pyy + pzz * pzz +
                          2.0f * (pxy * pxy + pxz * pxz + pyz * pyz));
    // tau - tau0 without cancellation: X / (2 (s + tau0)), s = sqrt(tau0^2 + X)
    const float X = kp.A * q * irho;
    const float s = csqrt<SCALED>(kp.tau0 * kp.tau0 + X);
    const float dtau = cdiv<SCALED>(0.5f * X, s + kp.tau0);
    const float om = crcp<SCALED>(kp.tau0 + dtau);
    const float keep = 1.0f - om;
    const float guo = 1.0f - 0.5f * om;
    const float uF = ux * Fx + uy * Fy + uz * Fz;
    // feq_i - w_i = w_i (drho + rho (3 cu + 4.5 cu^2 - 1.5 u.u)),
    // S_i = guo w_i (3 cF - 3 u.F + 9 cu cF)
    const float base = drho - 1.5f * rho * usq;       // even part of (feq - w)/w at cu = 0
    const float gbase = -3.0f * guo * uF;             // even part of S/w at cF = 0
    // node-wide coefficients, so that each direction pair costs
    // even = w (A0 + cu (Bq cu + Cq cF)), odd = w (Dq cu + Eq cF)
    // (A0 = om base + gbase; measured 1-2 % faster than expanding the terms
    // per direction)
    const float A0 = om * base + gbase;
    const float Bq = 4.5f * om * rho, Cq = 9.0f * guo;
    const float Dq = 3.0f * om * rho, Eq = 3.0f * guo;
    const float wa = sf * w19(1), wd = sf * w19(7);
    f[0] = keep * f[0] + sf * w19(0) * A0;
#pragma unroll
    for (int i = 1; i < 19; i += 2) {
        const float cu = cx27(i) * ux + cy27(i) * uy + cz27(i) * uz;
        const float cF = cx27(i) * Fx + cy27(i) * Fy + cz27(i) * Fz;
        const float w = i < 7 ? wa : wd;
        const float even = w * fmaf(cu, fmaf(Bq, cu, Cq * cF), A0);
        const float odd = w * fmaf(Dq, cu, Eq * cF);
        f[i] = fmaf(keep, f[i], even + odd);
        f[i + 1] = fmaf(keep, f[i + 1], even - odd);
    }

    const float omp = crcp<SCALED>(kp.taup0 + kp.kT * dtau);
    if constexpr (SL == 7) {
        // scalar: Phi_eq - w = w (chi - 1 + 4 chi c.u).  Only the non-equilibrium
        // parts are relaxed, and the rest population's part closes their sum to
        // zero, so the update conserves sum Phi exactly up to the rounding of the
        // stored results (relaxing towards the rounded chi would inject
        // omega times the rounding error of the 7-term sum at every node)
        const float pe = w7(1) * chs, pa = sp * w7(1) * 4.0f * chi;
        float nq[7];
        nq[1] = p[1] - (pe + pa * ux);
        nq[2] = p[2] - (pe - pa * ux);
        nq[3] = p[3] - (pe + pa * uy);
        nq[4] = p[4] - (pe - pa * uy);
        nq[5] = p[5] - (pe + pa * uz);
        nq[6] = p[6] - (pe - pa * uz);
        nq[0] = -(((nq[1] + nq[2]) + (nq[3] + nq[4])) + (nq[5] + nq[6]));
#pragma unroll
        for (int k = 0; k < 7; ++k) p[k] -= omp * nq[k];
    } else {
        // D3Q6: Phi_eq - w = (chi - 1 + 3 chi c.u) / 6; with no rest population
        // the non-equilibrium parts are centred on their mean instead
        const float pe = chs * (1.0f / 6.0f), pa = sp * 0.5f * chi;
        float nq[6];
        nq[0] = p[0] - (pe + pa * ux);
        nq[1] = p[1] - (pe - pa * ux);
        nq[2] = p[2] - (pe + pa * uy);
        nq[3] = p[3] - (pe - pa * uy);
        nq[4] = p[4] - (pe + pa * uz);
        nq[5] = p[5] - (pe - pa * uz);
        const float r = (((nq[0] + nq[1]) + (nq[2] + nq[3])) + (nq[4] + nq[5])) * (1.0f / 6.0f);
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k] -= omp * (nq[k] - r);
    }
}

}  // namespace lbmgpu
