// lbm_adjoint.cu -- discrete adjoint of the BGK-Smagorinsky + scalar +
// Boussinesq step, and the out-of-place forward step that recomputes the
// trajectory for it.  The objective is the time-integrated bottom friction
// J = sum_n F_w(s_n) (Eq. 62-64); the step differentiated is Eq. 11, 17,
// 19-30 and 32-35 as computed by collide_bgk.
#include "lbm_aa2.cuh"
#include "lbm_bgk_collide.cuh"
#include "lbm_internal.h"

namespace lbmgpu {

// ---------------------------------------------------------------------------
// Out-of-place step on the canonical FP32 layout (f - w, Phi - w), used to
// recompute the forward trajectory inside the adjoint sweep: each node reads
// its own populations at step n, collides, and pushes post-collision value i
// to slot i of node x + c_i, or to slot opp(i) of itself across a wall
// (Eq. 17).  Same arithmetic as the AA kernels, 208 bytes per node.
__global__ void __launch_bounds__(128, LBM_STEP_MINB) bgk_push_kernel(KParams kp,
                                                                      const float* __restrict__ src,
                                                                      float* __restrict__ dst) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= kp.nx) return;
    const Stencil st = make_stencil(kp, x, blockIdx.y, blockIdx.z);
    const unsigned n = st.n, N = kp.N;
    float f[19], p[7];
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = ld_chk(kp, LBM_SITE_ADJOINT, src, (unsigned)i * N + n, (size_t)26 * N);
#pragma unroll
    for (int k = 0; k < 7; ++k) p[k] = ld_chk(kp, LBM_SITE_ADJOINT, src, (unsigned)(19 + k) * N + n, (size_t)26 * N);
    if (!(kp.flags & LBM_FLAG_NO_COLLIDE)) collide_bgk(kp, f, p);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        bool in = false;
        const unsigned d = i == 0 ? n : nbr(st, cx27(i), cy27(i), cz27(i), in);
        st_chk(kp, LBM_SITE_ADJOINT, dst, (i != 0 && in) ? (unsigned)i * N + d : (unsigned)opp(i) * N + n,
               (size_t)26 * N, f[i]);
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        bool in = false;
        const unsigned d = k == 0 ? n : nbr(st, cx27(k), cy27(k), cz27(k), in);
        st_chk(kp, LBM_SITE_ADJOINT, dst,
               (k != 0 && in) ? (unsigned)(19 + k) * N + d : (unsigned)(19 + opp(k)) * N + n,
               (size_t)26 * N, p[k]);
    }
}

// The same push for two x-adjacent nodes per thread (nx even): reading the
// own slots is the AA even-step gather and pushing to slot i of node x + c_i
// (own slot opp(i) across a wall) is the AA odd-step scatter, both with
// paired accesses (lbm_aa2.cuh), here between two arrays.
template <bool ZW>
__device__ __forceinline__ void bgk_push2_body(const KParams& kp, const float* __restrict__ src,
                                               float* __restrict__ dst, const Stencil2& st) {
    const unsigned N = kp.N;
    float f0[19], f1[19], p0[7], p1[7];
    gather2<19, false>(kp, src, st, f0, f1);
    gather2<7, false>(kp, src + (size_t)19 * N, st, p0, p1);
    if (!(kp.flags & LBM_FLAG_NO_COLLIDE)) {
        collide_bgk(kp, f0, p0);
        collide_bgk(kp, f1, p1);
    }
    scatter2<19, true, float, 0, false, ZW>(kp, dst, st, f0, f1);
    scatter2<7, true, float, 0, false, ZW>(kp, dst + (size_t)19 * N, st, p0, p1);
}

__global__ void __launch_bounds__(128, LBM_STEP2_MINB) bgk_push2_kernel(KParams kp,
                                                                      const float* __restrict__ src,
                                                                      float* __restrict__ dst) {
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const Stencil2 st = make_stencil2(kp, x, blockIdx.y, blockIdx.z);
    const int z = blockIdx.z;
    // rows away from the z walls (uniform per block) skip the wall selects
    if ((kp.flags & LBM_FLAG_PERIODIC_Z) || (z > 0 && z < kp.nz - 1))
        bgk_push2_body<false>(kp, src, dst, st);
    else
        bgk_push2_body<true>(kp, src, dst, st);
}

cudaError_t launch_push_step(const KParams& kp, const float* src, float* dst, cudaStream_t st) {
    if (kp.nx % 2 == 0) {
        dim3 block(128), grid((kp.nx / 2 + 127) / 128, kp.ny, kp.nz);
        bgk_push2_kernel<<<grid, block, 0, st>>>(kp, src, dst);
        return cudaGetLastError();
    }
    dim3 block(128), grid((kp.nx + 127) / 128, kp.ny, kp.nz);
    bgk_push_kernel<<<grid, block, 0, st>>>(kp, src, dst);
    return cudaGetLastError();
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
// Minimum resident blocks per SM requested from the register allocator: 6
// caps the kernel at 80 registers (44 bytes of spills, served by L1) for 24
// resident warps per SM; measured faster than 4 (128 registers) and 5 (96).
#ifndef LBM_ADJ_MINB
#define LBM_ADJ_MINB 6
#endif

__global__ void __launch_bounds__(128, LBM_ADJ_MINB) bgk_adjoint_kernel(KParams kp, const float* __restrict__ st,
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
            mu[i] = lamn ? ld_chk(kp, LBM_SITE_ADJOINT, lamn, off, (size_t)26 * N) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            bool in = false;
            const unsigned d = k == 0 ? n : nbr(sn, cx27(k), cy27(k), cz27(k), in);
            const unsigned off = (k != 0 && in) ? (unsigned)(19 + k) * N32 + d
                                                : (unsigned)(19 + opp(k)) * N32 + n;
            mup[k] = lamn ? ld_chk(kp, LBM_SITE_ADJOINT, lamn, off, (size_t)26 * N) : 0.0f;
        }
        float f[19], p[7];
#pragma unroll
        for (int i = 0; i < 19; ++i) f[i] = ld_chk(kp, LBM_SITE_ADJOINT, st, (size_t)i * N + n, (size_t)26 * N);
#pragma unroll
        for (int k = 0; k < 7; ++k) p[k] = ld_chk(kp, LBM_SITE_ADJOINT, st, (size_t)(19 + k) * N + n, (size_t)26 * N);

        // ---- forward recompute (as collide_bgk) ----
        float chit = 0.0f;
#pragma unroll
        for (int k = 0; k < 7; ++k) chit += p[k];
        const float chi = 1.0f + chit;
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
        // fluid: f* = (1 - om) f + om feq + (1 - om/2) B, with
        //   feq_i = w_i (drho + rho (3 cu + 4.5 cu^2 - 1.5 u.u)),
        //   B_i = w_i (3 cF - 3 u.F + 9 cu cF),  cu = c_i.u, cF = c_i.F.
        // Both are polynomials of degree 2 in c_i, so every sum over i of mu_i
        // times them or their derivatives is a combination of the weighted
        // moments of the adjoint A0 = sum w mu, A1 = sum w mu c, A2 = sum w mu c c
        // (taken with opposite-pair sums and differences):
        //   sum mu feq = drho A0 + rho (3 u.A1 + 4.5 u.A2.u - 1.5 u.u A0)
        //   sum mu B   = 3 F.A1 - 3 u.F A0 + 9 u.A2.F
        //   d/d drho   : om (A0 + 3 u.A1 + 4.5 u.A2.u - 1.5 u.u A0)
        //   d/d u      : om rho V + guo (9 A2.F - 3 F A0),  V = 3 A1 + 9 A2.u - 3 u A0
        //   d/d F      : guo V
        float A0 = w19(0) * mu[0], A1x = 0.0f, A1y = 0.0f, A1z = 0.0f;
        float Axx = 0.0f, Ayy = 0.0f, Azz = 0.0f, Axy = 0.0f, Axz = 0.0f, Ayz = 0.0f;
        float muf = mu[0] * f[0];
        gf[0] = (1.0f - om) * mu[0];
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            const float w = w19(i);
            const float ms = w * (mu[i] + mu[i + 1]), md = w * (mu[i] - mu[i + 1]);
            muf += mu[i] * f[i] + mu[i + 1] * f[i + 1];
            A0 += ms;
            if (cx27(i)) { A1x += cx27(i) * md; Axx += ms; }
            if (cy27(i)) { A1y += cy27(i) * md; Ayy += ms; }
            if (cz27(i)) { A1z += cz27(i) * md; Azz += ms; }
            if (cx27(i) * cy27(i)) Axy += cx27(i) * cy27(i) * ms;
            if (cx27(i) * cz27(i)) Axz += cx27(i) * cz27(i) * ms;
            if (cy27(i) * cz27(i)) Ayz += cy27(i) * cz27(i) * ms;
            gf[i] = (1.0f - om) * mu[i];
            gf[i + 1] = (1.0f - om) * mu[i + 1];
        }
        const float Aux = Axx * ux + Axy * uy + Axz * uz;
        const float Auy = Axy * ux + Ayy * uy + Ayz * uz;
        const float Auz = Axz * ux + Ayz * uy + Azz * uz;
        const float AFx = Axx * Fx + Axy * Fy + Axz * Fz;
        const float AFy = Axy * Fx + Ayy * Fy + Ayz * Fz;
        const float AFz = Axz * Fx + Ayz * Fy + Azz * Fz;
        const float uA1 = ux * A1x + uy * A1y + uz * A1z;
        const float uAu = ux * Aux + uy * Auy + uz * Auz;
        const float FA1 = Fx * A1x + Fy * A1y + Fz * A1z;
        const float uAF = ux * AFx + uy * AFy + uz * AFz;
        const float pe = 3.0f * uA1 + 4.5f * uAu - 1.5f * usq * A0;
        const float gom = drho * A0 + rho * pe - muf - 0.5f * (3.0f * FA1 - 3.0f * uF * A0 + 9.0f * uAF);
        grho += om * (A0 + pe);
        const float Vx = 3.0f * A1x + 9.0f * Aux - 3.0f * ux * A0;
        const float Vy = 3.0f * A1y + 9.0f * Auy - 3.0f * uy * A0;
        const float Vz = 3.0f * A1z + 9.0f * Auz - 3.0f * uz * A0;
        const float orho = om * rho;
        gux += orho * Vx + guo * (9.0f * AFx - 3.0f * Fx * A0);
        guy += orho * Vy + guo * (9.0f * AFy - 3.0f * Fy * A0);
        guz += orho * Vz + guo * (9.0f * AFz - 3.0f * Fz * A0);
        gFx += guo * Vx; gFy += guo * Vy; gFz += guo * Vz;
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
        // (even part grho + c c : gP, odd part c . gj for each opposite pair)
        gf[0] += grho;
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            const float cxi = cx27(i), cyi = cy27(i), czi = cz27(i);
            const float te = grho + gpxx * cxi * cxi + gpyy * cyi * cyi + gpzz * czi * czi +
                             gpxy * cxi * cyi + gpxz * cxi * czi + gpyz * cyi * czi;
            const float to = cxi * gjx + cyi * gjy + czi * gjz;
            gf[i] += te + to;
            gf[i + 1] += te - to;
        }
        // F = g' chi e^g, chi = 1 + sum (Phi - w)
        gchi += gFx * kp.gx + gFy * kp.gy + gFz * kp.gz;
#pragma unroll
        for (int k = 0; k < 7; ++k) gp[k] += gchi;
#pragma unroll
        for (int i = 0; i < 19; ++i) st_chk(kp, LBM_SITE_ADJOINT, lam, (size_t)i * N + n, (size_t)26 * N, gf[i]);
#pragma unroll
        for (int k = 0; k < 7; ++k) st_chk(kp, LBM_SITE_ADJOINT, lam, (size_t)(19 + k) * N + n, (size_t)26 * N, gp[k]);
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
