// lbm_adjoint_cumulant.cu -- discrete adjoint of the D3Q27 cumulant + D3Q7
// scalar + Boussinesq step (collide_cumulant<7>, Eq. 54-58 with every rate of
// order >= 3 equal to 1, and Eq. 28-30 with the molecular D), and the
// out-of-place forward step that recomputes the trajectory for it.
#include "lbm_cumulant_collide.cuh"
#include "lbm_internal.h"

// Minimum resident blocks per SM for the adjoint kernel's register allocation:
// 3 (168 registers) measured a reverse step 4 % shorter than 4 (128
// registers, 84 bytes of spills) on the 256x32x64 box.
#ifndef LBM_CUM_ADJ_MINB
#define LBM_CUM_ADJ_MINB 3
#endif

namespace lbmgpu {

// Out-of-place step on the canonical FP32 layout: the own slots are read as
// on an even AA step and each post-collision population is pushed to slot i
// of node x + c_i (own slot opp(i) across a wall) as on an odd AA step.
// Element offsets of the saved state and the adjoint field: 32-bit (the
// adjoint entry points need (Q + NS) N < 2^32); at 168 registers they spill
// nothing (64-bit: 8 bytes) and the reverse step took 1.2 % less time.
#ifndef LBM_CUM_ADJ_OFF
#define LBM_CUM_ADJ_OFF unsigned
#endif
// The recompute kernel keeps the compiler's register choice (72, no spills):
// 5 to 8 resident blocks with 32- or 64-bit offsets measured 2-3 % slower
// reverse steps.
#ifndef LBM_CUM_PUSH_MINB
#define LBM_CUM_PUSH_MINB 0
#endif
#if LBM_CUM_PUSH_MINB
#define LBM_CUM_PUSH_BOUNDS __launch_bounds__(128, LBM_CUM_PUSH_MINB)
#else
#define LBM_CUM_PUSH_BOUNDS __launch_bounds__(128)
#endif
#ifndef LBM_CUM_PUSH_OFF
#define LBM_CUM_PUSH_OFF unsigned
#endif
__global__ void LBM_CUM_PUSH_BOUNDS cumulant_push_kernel(KParams kp, const float* __restrict__ src,
                                                            float* __restrict__ dst) {
    using Off = LBM_CUM_PUSH_OFF;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const Stencil st = make_stencil(kp, x, blockIdx.y, blockIdx.z);
    const size_t N = kp.N;
    float f[27], p[7];
    gather<27, false, float, 0, false, true, Off>(kp, src, st, f);
    gather<7, false, float, 0, false, true, Off>(kp, src + 27 * N, st, p);
    if (!(kp.flags & LBM_FLAG_NO_COLLIDE)) collide_cumulant<7>(kp, f, p);
    scatter<27, true, float, 0, false, true, Off>(kp, dst, st, f);
    scatter<7, true, float, 0, false, true, Off>(kp, dst + 27 * N, st, p);
}

cudaError_t launch_cumulant_push_step(const KParams& kp, const float* src, float* dst,
                                      cudaStream_t st) {
    dim3 block(128), grid((kp.nx + 127) / 128, kp.ny, kp.nz);
    cumulant_push_kernel<<<grid, block, 0, st>>>(kp, src, dst);
    return cudaGetLastError();
}

// Reverse of axis_inverse: from the adjoints (gm, g0, gp) of the outputs
// (p(-1), p(0), p(+1)) to those of the inputs (d0, d1, d2); adds the adjoint
// of the frame velocity v to gv.  With k0 = s + d0, a = v^2 k0 + 2 v d1 + d2,
// b = v k0 + d1: p(0) = d0 - k0 v^2 - 2 v d1 - d2, p(+-1) = (a +- b) / 2.
__device__ __forceinline__ void axis_inverse_vjp(float s, float v, float d0, float d1, float gm,
                                                 float g0, float gp, float& gd0, float& gd1,
                                                 float& gd2, float& gv) {
    const float k0 = s + d0;
    const float ga = 0.5f * (gp + gm), gb = 0.5f * (gp - gm);
    const float v2 = v * v;
    gd0 = g0 * (1.0f - v2) + ga * v2 + gb * v;
    gd1 = 2.0f * v * (ga - g0) + gb;
    gd2 = ga - g0;
    gv += 2.0f * (v * k0 + d1) * (ga - g0) + gb * k0;
}

// The same, also adding to dot the value of sum_j g_j p(j) over the line's
// outputs, gm p(-1) + g0 p(0) + gp p(+1), which for this affine stage is
// gd . (d0, d1, d2) + s ((ga - g0) v^2 + gb v) (d2: the line's third input).
__device__ __forceinline__ void axis_inverse_vjp(float s, float v, float d0, float d1, float gm,
                                                 float g0, float gp, float& gd0, float& gd1,
                                                 float& gd2, float& gv, float d2, float& dot) {
    axis_inverse_vjp(s, v, d0, d1, gm, g0, gp, gd0, gd1, gd2, gv);
    const float ga = 0.5f * (gp + gm), gb = 0.5f * (gp - gm);
    dot += gd0 * d0 + gd1 * d1 + gd2 * d2 + s * ((ga - g0) * (v * v) + gb * v);
}

// One reverse step: lam_n = C(s_n)^T P^T lam_{n+1} + w_fw dF_w/ds_n, with P^T
// reading lam_{n+1} where each post-collision population was pushed and C^T
// the reverse-mode derivative of collide_cumulant<7> written out by hand
// (in exact arithmetic the rest populations' closing sums equal their
// formulas, which are what is differentiated).  The cumulant model has no
// Smagorinsky closure, so there is no C_s term.
__global__ void __launch_bounds__(128, LBM_CUM_ADJ_MINB) cumulant_adjoint_kernel(KParams kp, const float* __restrict__ st,
                                                               const float* __restrict__ lamn,
                                                               float* __restrict__ lam, float wfw) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const Stencil sn = make_stencil(kp, x, y, z);
    const unsigned n = sn.n, N = kp.N;
    float mu[27], mup[7];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        bool in = false;
        const unsigned d = i == 0 ? n : nbr(sn, cx27(i), cy27(i), cz27(i), in);
        const unsigned off = (i != 0 && in) ? (unsigned)i * N + d : (unsigned)opp(i) * N + n;
        mu[i] = lamn ? ld_chk(kp, LBM_SITE_ADJOINT, lamn, off, (size_t)34 * N) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        bool in = false;
        const unsigned d = k == 0 ? n : nbr(sn, cx27(k), cy27(k), cz27(k), in);
        const unsigned off = (k != 0 && in) ? (unsigned)(27 + k) * N + d : (unsigned)(27 + opp(k)) * N + n;
        mup[k] = lamn ? ld_chk(kp, LBM_SITE_ADJOINT, lamn, off, (size_t)34 * N) : 0.0f;
    }
    float f[27], p[7];
#pragma unroll
    for (int i = 0; i < 27; ++i) f[i] = ld_chk(kp, LBM_SITE_ADJOINT, st, (LBM_CUM_ADJ_OFF)i * N + n, (size_t)34 * N);
#pragma unroll
    for (int k = 0; k < 7; ++k) p[k] = ld_chk(kp, LBM_SITE_ADJOINT, st, (LBM_CUM_ADJ_OFF)(27 + k) * N + n, (size_t)34 * N);

    // ---- forward recompute (as collide_cumulant<7>) ----
    float chit = 0.0f;
#pragma unroll
    for (int k = 0; k < 7; ++k) chit += p[k];
    const float chi = 1.0f + chit;
    const float Fx = kp.gx * chi, Fy = kp.gy * chi, Fz = kp.gz * chi;
    // the forward's moments, summed by lines as it sums them
    const Moments2 mo = moments_by_lines(f);
    const float drho = mo.drho, jx = mo.jx, jy = mo.jy, jz = mo.jz;
    const float mxx = mo.mxx, myy = mo.myy, mzz = mo.mzz, mxy = mo.mxy, mxz = mo.mxz,
                myz = mo.myz;
    const float rho = 1.0f + drho, irho = 1.0f / rho;
    const float vx = jx * irho, vy = jy * irho, vz = jz * irho;
    const float d3 = drho * (1.0f / 3.0f);
    const float cxx = (mxx - d3) * irho - vx * vx;
    const float cyy = (myy - d3) * irho - vy * vy;
    const float czz = (mzz - d3) * irho - vz * vz;
    const float cxy = mxy * irho - vx * vy;
    const float cxz = mxz * irho - vx * vz;
    const float cyz = myz * irho - vy * vz;
    const float r1 = 1.0f - kp.om1, r2 = 1.0f - kp.om2;
    const float D1 = r1 * (cxx - cyy), D2 = r1 * (cxx - czz), T = r2 * (cxx + cyy + czz);
    const float sxx = (T + D1 + D2) * (1.0f / 3.0f);
    const float syy = sxx - D1, szz = sxx - D2;
    const float sxy = r1 * cxy, sxz = r1 * cxz, syz = r1 * cyz;
    const float ux = (jx + Fx) * irho, uy = (jy + Fy) * irho, uz = (jz + Fz) * irho;
    const float t3 = 1.0f / 3.0f;
    const float sgx = t3 + sxx, sgy = t3 + syy, sgz = t3 + szz;
    float K[3][3][3];
#pragma unroll
    for (int a = 0; a < 27; ++a) (&K[0][0][0])[a] = 0.0f;
    K[2][0][0] = sxx; K[0][2][0] = syy; K[0][0][2] = szz;
    K[1][1][0] = sxy; K[1][0][1] = sxz; K[0][1][1] = syz;
    K[2][2][0] = (sxx + syy) * t3 + sxx * syy + 2.0f * sxy * sxy;
    K[2][0][2] = (sxx + szz) * t3 + sxx * szz + 2.0f * sxz * sxz;
    K[0][2][2] = (syy + szz) * t3 + syy * szz + 2.0f * syz * syz;
    K[2][1][1] = sgx * syz + 2.0f * sxy * sxz;
    K[1][2][1] = sgy * sxz + 2.0f * sxy * syz;
    K[1][1][2] = sgz * sxy + 2.0f * sxz * syz;
    K[2][2][2] = (sxx + syy + szz) * (1.0f / 9.0f) + (sxx * syy + sxx * szz + syy * szz) * t3 +
                 sxx * syy * szz + 2.0f * (sgx * syz * syz + sgy * sxz * sxz + sgz * sxy * sxy) +
                 8.0f * sxy * sxz * syz;
    constexpr float R[3] = {1.0f, 0.0f, 1.0f / 3.0f};
    constexpr float W1[3] = {1.0f / 6.0f, 2.0f / 3.0f, 1.0f / 6.0f};
    float A[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            axis_inverse(R[a] * R[b], uz, K[a][b][0], K[a][b][1], K[a][b][2], A[a][b][0],
                         A[a][b][1], A[a][b][2]);
    float B[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            axis_inverse(R[a] * W1[c], uy, A[a][0][c], A[a][1][c], A[a][2][c], B[a][0][c],
                         B[a][1][c], B[a][2][c]);
    const float hx = (jx + 0.5f * Fx) * irho, hy = (jy + 0.5f * Fy) * irho,
                hz = (jz + 0.5f * Fz) * irho;
    // equal to kp.omp0 bit for bit (both the IEEE quotient); the division
    // schedules better here than the parameter load (the kernel runs 12 % faster)
    const float omp = 1.0f / kp.taup0;

    // ---- reverse ----
    // f*_i - w_i = drho w_i + rho P_i with P_i the deviations the x-stage
    // returns, so d/d drho = sum_i mu_i (w_i + P_i).  The x-stage is affine
    // in its line (d0, d1, d2) with the rest offset s, so sum over a line of
    // mu P = (gd . d + s ((ga - g0) v^2 + gb v)) / rho for the adjoints gd the
    // stage's reverse returns from (rho mu): no forward x-stage is needed.
    float gux = 0.0f, guy = 0.0f, guz = 0.0f, smuP = 0.0f;
    float gB[3][3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int im = dir27(-1, b - 1, c - 1), i0 = dir27(0, b - 1, c - 1),
                      ip = dir27(1, b - 1, c - 1);
            axis_inverse_vjp(W1[b] * W1[c], ux, B[0][b][c], B[1][b][c], rho * mu[im], rho * mu[i0],
                             rho * mu[ip], gB[0][b][c], gB[1][b][c], gB[2][b][c], gux,
                             B[2][b][c], smuP);
        }
    float gdrho = smuP * irho;
#pragma unroll
    for (int i = 0; i < 27; ++i) gdrho += w27(i) * mu[i];
    float gA[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            axis_inverse_vjp(R[a] * W1[c], uy, A[a][0][c], A[a][1][c], gB[a][0][c], gB[a][1][c],
                             gB[a][2][c], gA[a][0][c], gA[a][1][c], gA[a][2][c], guy);
    float gK[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            axis_inverse_vjp(R[a] * R[b], uz, K[a][b][0], K[a][b][1], gA[a][b][0], gA[a][b][1],
                             gA[a][b][2], gK[a][b][0], gK[a][b][1], gK[a][b][2], guz);
    // Gaussian moments -> relaxed covariance deviations s
    const float g222 = gK[2][2][2];
    const float gsxx = gK[2][0][0] + gK[2][2][0] * (t3 + syy) + gK[2][0][2] * (t3 + szz) +
                       gK[2][1][1] * syz +
                       g222 * ((1.0f / 9.0f) + (syy + szz) * t3 + syy * szz + 2.0f * syz * syz);
    const float gsyy = gK[0][2][0] + gK[2][2][0] * (t3 + sxx) + gK[0][2][2] * (t3 + szz) +
                       gK[1][2][1] * sxz +
                       g222 * ((1.0f / 9.0f) + (sxx + szz) * t3 + sxx * szz + 2.0f * sxz * sxz);
    const float gszz = gK[0][0][2] + gK[2][0][2] * (t3 + sxx) + gK[0][2][2] * (t3 + syy) +
                       gK[1][1][2] * sxy +
                       g222 * ((1.0f / 9.0f) + (sxx + syy) * t3 + sxx * syy + 2.0f * sxy * sxy);
    const float gsxy = gK[1][1][0] + gK[2][2][0] * 4.0f * sxy + gK[2][1][1] * 2.0f * sxz +
                       gK[1][2][1] * 2.0f * syz + gK[1][1][2] * sgz +
                       g222 * (4.0f * sgz * sxy + 8.0f * sxz * syz);
    const float gsxz = gK[1][0][1] + gK[2][0][2] * 4.0f * sxz + gK[2][1][1] * 2.0f * sxy +
                       gK[1][2][1] * sgy + gK[1][1][2] * 2.0f * syz +
                       g222 * (4.0f * sgy * sxz + 8.0f * sxy * syz);
    const float gsyz = gK[0][1][1] + gK[0][2][2] * 4.0f * syz + gK[2][1][1] * sgx +
                       gK[1][2][1] * 2.0f * sxy + gK[1][1][2] * 2.0f * sxz +
                       g222 * (4.0f * sgx * syz + 8.0f * sxy * sxz);
    // relaxation: s from the pre-collision covariance deviations c
    const float G = (gsxx + gsyy + gszz) * t3;
    const float gD1 = G - gsyy, gD2 = G - gszz;
    const float gcxx = r1 * (gD1 + gD2) + r2 * G;
    const float gcyy = -r1 * gD1 + r2 * G;
    const float gczz = -r1 * gD2 + r2 * G;
    const float gcxy = r1 * gsxy, gcxz = r1 * gsxz, gcyz = r1 * gsyz;
    // c from the moments: c_aa = (m_aa - drho/3)/rho - v_a^2, c_ab = m_ab/rho - v_a v_b
    const float gmxx = gcxx * irho, gmyy = gcyy * irho, gmzz = gczz * irho;
    const float gmxy = gcxy * irho, gmxz = gcxz * irho, gmyz = gcyz * irho;
    gdrho += -(gcxx + gcyy + gczz) * irho * (1.0f / 3.0f);
    float girho = gcxx * (mxx - d3) + gcyy * (myy - d3) + gczz * (mzz - d3) + gcxy * mxy +
                  gcxz * mxz + gcyz * myz;
    const float gvx = -2.0f * vx * gcxx - vy * gcxy - vz * gcxz;
    const float gvy = -2.0f * vy * gcyy - vx * gcxy - vz * gcyz;
    const float gvz = -2.0f * vz * gczz - vx * gcxz - vy * gcyz;
    // scalar: Phi*_k = Phi_k - omp (Phi_k - w_k (chit + 4 chi c_k.h))
    float gp[7], gchit = 0.0f, ghx = 0.0f, ghy = 0.0f, ghz = 0.0f;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const float ch = cx27(k) * hx + cy27(k) * hy + cz27(k) * hz;
        gp[k] = (1.0f - omp) * mup[k];
        const float g = omp * mup[k] * w7(k);
        gchit += g * (1.0f + 4.0f * ch);
        const float a = g * 4.0f * chi;
        ghx += a * cx27(k); ghy += a * cy27(k); ghz += a * cz27(k);
    }
    // objective: F_w = sum_{x,y} nu (9 u_x(z=0) - u_x(z=1)) / 3 with the half-force u (Eq. 62-64)
    if (wfw != 0.0f && kp.nz >= 2) {
        if (z == 0) ghx += wfw * 3.0f * kp.nu;
        else if (z == 1) ghx += -wfw * kp.nu * (1.0f / 3.0f);
    }
    // v = j / rho, u = (j + F) / rho, h = (j + F/2) / rho
    const float gjx = (gvx + gux + ghx) * irho, gjy = (gvy + guy + ghy) * irho,
                gjz = (gvz + guz + ghz) * irho;
    const float gFx = (gux + 0.5f * ghx) * irho, gFy = (guy + 0.5f * ghy) * irho,
                gFz = (guz + 0.5f * ghz) * irho;
    girho += gvx * jx + gvy * jy + gvz * jz + gux * (jx + Fx) + guy * (jy + Fy) + guz * (jz + Fz) +
             ghx * (jx + 0.5f * Fx) + ghy * (jy + 0.5f * Fy) + ghz * (jz + 0.5f * Fz);
    gdrho += -girho * irho * irho;
    // F = g' chi e^g
    gchit += gFx * kp.gx + gFy * kp.gy + gFz * kp.gz;
    // f enters through drho, j and the second moments
    // d/df_i of the moments: gdrho + c.gj + sum_ab c_a c_b gm_ab, built by
    // lines (49 operations): E, the part without c_x, and X, the coefficient
    // of c_x, per (c_y, c_z), then E (c_x = 0) and E + gmxx +- X (c_x = +-1)
    const float u = gdrho + gmzz;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float Ez = c == 1 ? gdrho : (c == 2 ? u + gjz : u - gjz);
        const float Xz = c == 1 ? gjx : (c == 2 ? gjx + gmxz : gjx - gmxz);
        const float Yz = c == 1 ? gjy : (c == 2 ? gjy + gmyz : gjy - gmyz);
        const float t = Ez + gmyy;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float E = b == 1 ? Ez : (b == 2 ? t + Yz : t - Yz);
            const float X = b == 1 ? Xz : (b == 2 ? Xz + gmxy : Xz - gmxy);
            const float gx = E + gmxx;
            st_chk(kp, LBM_SITE_ADJOINT, lam, (LBM_CUM_ADJ_OFF)dir27(-1, b - 1, c - 1) * N + n, (size_t)34 * N, gx - X);
            st_chk(kp, LBM_SITE_ADJOINT, lam, (LBM_CUM_ADJ_OFF)dir27(0, b - 1, c - 1) * N + n, (size_t)34 * N, E);
            st_chk(kp, LBM_SITE_ADJOINT, lam, (LBM_CUM_ADJ_OFF)dir27(1, b - 1, c - 1) * N + n, (size_t)34 * N, gx + X);
        }
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) st_chk(kp, LBM_SITE_ADJOINT, lam, (LBM_CUM_ADJ_OFF)(27 + k) * N + n, (size_t)34 * N, gp[k] + gchit);
}

cudaError_t launch_cumulant_adjoint_step(const KParams& kp, const float* state,
                                         const float* lam_next, float* lam, float wfw,
                                         cudaStream_t st) {
    dim3 block(128), grid((kp.nx + 127) / 128, kp.ny, kp.nz);
    cumulant_adjoint_kernel<<<grid, block, 0, st>>>(kp, state, lam_next, lam, wfw);
    return cudaGetLastError();
}

}  // namespace lbmgpu
