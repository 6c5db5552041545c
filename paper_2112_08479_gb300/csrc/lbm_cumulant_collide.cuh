// lbm_cumulant_collide.cuh -- the per-node collision of the D3Q27 cumulant
// fluid with the D3Q7 or D3Q27 scalar and the Boussinesq force, shared by the
// AA step kernel, the out-of-place recompute and the adjoint.
//
// Cumulants C_abc are the derivatives of ln G, G(Xi) = sum_i f_i exp(Xi.c_i)
// (Eq. 54).  The collision keeps rho (Eq. 56), moves the first-order
// cumulants to u* = (j + F) / rho (Eq. 57 plus the body-force impulse),
// relaxes the second-order ones with omega1 = 1/(3 nu + 1/2) (Eq. 58) on
// the shear parts and omega_bulk on the trace (Eq. 55, C_eq = c_s^2 = 1/3
// per axis), and relaxes every cumulant of order >= 3 with rate 1 to its
// equilibrium 0.  Because all higher cumulants leave the collision as 0,
// only the pre-collision moments of order <= 2 are needed, and the
// post-collision distribution has the truncated moment generating function
//   G* = rho exp(u*.Xi) exp(Xi^T Sigma* Xi / 2)   mod (Xi^3, Y^3, Z^3),
// whose central moments are rho times the Gaussian moments of Sigma*
// (Isserlis): kappa_220 = s_xx s_yy + 2 s_xy^2, kappa_211 = s_xx s_yz +
// 2 s_xy s_xz, kappa_222 = s_xx s_yy s_zz + 2 (s_xx s_yz^2 + s_yy s_xz^2 +
// s_zz s_xy^2) + 8 s_xy s_xz s_yz, odd orders 0.  The populations follow from
// the per-axis inverse of the central-moment map in the frame u*, applied on
// z, then y, then x.  Every quantity is carried as a deviation from the rest
// state (rho = 1, u = 0, Sigma = I/3) so FP32 keeps its digits.
#pragma once

#include "lbm_common.cuh"

namespace lbmgpu {

// Per-axis inverse of the central-moment map, in deviation form.  A line
// (k0, k1, k2) of central moments in the frame moving with v holds the rest
// values s * (1, 0, 1/3) plus the deviations (d0, d1, d2); the populations at
// c = -1, 0, +1 are the rest values s * (1/6, 2/3, 1/6) plus the returned
// deviations:
//   p(0)  = d0 - (s + d0) v^2 - 2 v d1 - d2 = d0 - a
//   p(+-) = ((v^2 +- v)(s + d0) + (2 v +- 1) d1 + d2) / 2 = (a +- b) / 2
// with a = (s + d0) v^2 + 2 v d1 + d2 and b = (s + d0) v + d1.
__device__ __forceinline__ void axis_inverse(float s, float v, float d0, float d1, float d2,
                                             float& pm, float& p0, float& pp) {
    const float k0 = s + d0;
    const float v2 = v * v;
    const float a = v2 * k0 + 2.0f * v * d1 + d2;
    const float b = v * k0 + d1;
    p0 = d0 - a;
    pp = 0.5f * (a + b);
    pm = 0.5f * (a - b);
}

// Index of the D3Q27 direction (cx, cy, cz) in the library order, looked up
// by (cx + 1) * 9 + (cy + 1) * 3 + (cz + 1).
__host__ __device__ constexpr int dir27(int x, int y, int z) {
    constexpr int t[27] = {20, 8, 22, 12, 2, 14, 24, 10, 25, 16, 4, 18, 6, 0,
                           5, 17, 3, 15, 26, 9, 23, 13, 1, 11, 21, 7, 19};
    return t[(x + 1) * 9 + (y + 1) * 3 + (z + 1)];
}

// Moments of order <= 2 of the 27 populations (held as f - w), summed by
// lines: along x for each (c_y, c_z), then along y for each c_z, then along
// z (66 additions; term by term the ten sums take 170).  drho = sum f,
// j = sum c f, m_ab = sum c_a c_b f.
struct Moments2 {
    float drho, jx, jy, jz, mxx, myy, mzz, mxy, mxz, myz;
};
__device__ __forceinline__ Moments2 moments_by_lines(const float (&f)[27]) {
    float L0[3][3], L1[3][3], L2[3][3];   // x-moments 0, 1, 2 of the line [cy + 1][cz + 1]
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float pm = f[dir27(-1, b - 1, c - 1)], p0 = f[dir27(0, b - 1, c - 1)],
                        pp = f[dir27(1, b - 1, c - 1)];
            L2[b][c] = pp + pm;
            L0[b][c] = L2[b][c] + p0;
            L1[b][c] = pp - pm;
        }
    float m00[3], m10[3], m01[3], m02[3], m11[3], m20[3];   // (x, y)-moments per cz + 1
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        m02[c] = L0[0][c] + L0[2][c];
        m00[c] = m02[c] + L0[1][c];
        m01[c] = L0[2][c] - L0[0][c];
        m10[c] = (L1[0][c] + L1[2][c]) + L1[1][c];
        m11[c] = L1[2][c] - L1[0][c];
        m20[c] = (L2[0][c] + L2[2][c]) + L2[1][c];
    }
    Moments2 m;
    m.mzz = m00[2] + m00[0];
    m.drho = m.mzz + m00[1];
    m.jx = (m10[0] + m10[2]) + m10[1];
    m.jy = (m01[0] + m01[2]) + m01[1];
    m.jz = m00[2] - m00[0];
    m.mxx = (m20[0] + m20[2]) + m20[1];
    m.myy = (m02[0] + m02[2]) + m02[1];
    m.mxy = (m11[0] + m11[2]) + m11[1];
    m.mxz = m10[2] - m10[0];
    m.myz = m01[2] - m01[0];
    return m;
}

// The fluid part: replaces f by its post-collision populations, given
// chs = sum_k (Phi_k - w_k) (storage units when SCALED); returns chi - 1,
// chi and the half-force velocity h = (j + F/2) / rho the scalar takes.
template <bool SCALED>
__device__ __forceinline__ void cumulant_fluid(const KParams& kp, float (&f)[27], float chs,
                                               float& chit_out, float& chi_out, float& hx,
                                               float& hy, float& hz) {
    const float chit = SCALED ? chs * kp.isp : chs;   // chi - chi_s
    const float chi = kp.chi_s + chit;
    const float Fx = kp.gx * chi, Fy = kp.gy * chi, Fz = kp.gz * chi;

    // moments of order <= 2, summed by lines
    const Moments2 mo = moments_by_lines(f);
    float drho = mo.drho, jx = mo.jx, jy = mo.jy, jz = mo.jz;
    float mxx = mo.mxx, myy = mo.myy, mzz = mo.mzz, mxy = mo.mxy, mxz = mo.mxz, myz = mo.myz;
    if (SCALED) {
        drho *= kp.isf; jx *= kp.isf; jy *= kp.isf; jz *= kp.isf;
        mxx *= kp.isf; myy *= kp.isf; mzz *= kp.isf; mxy *= kp.isf; mxz *= kp.isf; myz *= kp.isf;
    }
    const float rho = 1.0f + drho;
    const float irho = crcp<SCALED>(rho);
    // pre-collision mean velocity and second-order cumulants (deviation of
    // the diagonal from 1/3): C_aa - 1/3 = (M_aa - drho/3)/rho - v_a^2
    const float vx = jx * irho, vy = jy * irho, vz = jz * irho;
    const float d3 = drho * (1.0f / 3.0f);
    const float cxx = (mxx - d3) * irho - vx * vx;
    const float cyy = (myy - d3) * irho - vy * vy;
    const float czz = (mzz - d3) * irho - vz * vz;
    const float cxy = mxy * irho - vx * vy;
    const float cxz = mxz * irho - vx * vz;
    const float cyz = myz * irho - vy * vz;
    // relaxation (Eq. 55): shear with omega1, trace with omega_bulk
    const float r1 = 1.0f - kp.om1, r2 = 1.0f - kp.om2;
    const float D1 = r1 * (cxx - cyy), D2 = r1 * (cxx - czz), T = r2 * (cxx + cyy + czz);
    const float sxx = (T + D1 + D2) * (1.0f / 3.0f);
    const float syy = sxx - D1, szz = sxx - D2;
    const float sxy = r1 * cxy, sxz = r1 * cxz, syz = r1 * cyz;
    // post-collision velocity (first-order cumulants + body-force impulse)
    const float ux = (jx + Fx) * irho, uy = (jy + Fy) * irho, uz = (jz + Fz) * irho;

    // central-moment deviations K[a][b][c] (rho-normalised) of the Gaussian
    // with covariance I/3 + s; entries of odd total order vanish
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

    // rest value per moment order r = (1, 0, 1/3), per velocity w1 = (1/6, 2/3, 1/6)
    // for c = -1, 0, +1 (index c + 1)
    constexpr float R[3] = {1.0f, 0.0f, 1.0f / 3.0f};
    constexpr float W1[3] = {1.0f / 6.0f, 2.0f / 3.0f, 1.0f / 6.0f};
    float A[3][3][3];  // [a][b][cz + 1]
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            axis_inverse(R[a] * R[b], uz, K[a][b][0], K[a][b][1], K[a][b][2], A[a][b][0],
                         A[a][b][1], A[a][b][2]);
    float B[3][3][3];  // [a][cy + 1][cz + 1]
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            axis_inverse(R[a] * W1[c], uy, A[a][0][c], A[a][1][c], A[a][2][c], B[a][0][c],
                         B[a][1][c], B[a][2][c]);
    // f*_i - w_i = drho w_i + rho (P_i - w_i), in storage units when SCALED
    const float ds = SCALED ? drho * kp.sf : drho, rs = SCALED ? rho * kp.sf : rho;
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float pm, p0, pp;
            axis_inverse(W1[b] * W1[c], ux, B[0][b][c], B[1][b][c], B[2][b][c], pm, p0, pp);
            const int im = dir27(-1, b - 1, c - 1), i0 = dir27(0, b - 1, c - 1),
                      ip = dir27(1, b - 1, c - 1);
            f[im] = ds * w27(im) + rs * pm;
            f[i0] = ds * w27(i0) + rs * p0;
            f[ip] = ds * w27(ip) + rs * pp;
        }

    hx = (jx + 0.5f * Fx) * irho;
    hy = (jy + 0.5f * Fy) * irho;
    hz = (jz + 0.5f * Fz) * irho;
    chit_out = chit;
    chi_out = chi;
}

// Post-collision value of moving population i (1 .. 26) of the D3Q27
// factorized-central-moment scalar (collide_fcm27 below, one population):
// chi - 1, chi, the half-force velocity h and the relaxed first moments v.
struct Fcm27 {
    float chit, chi;
    float W[3][3], dE[3][3], G[3][3];   // [axis][c + 1]
    float v[3];
};
__device__ __forceinline__ Fcm27 fcm27_setup(const KParams& kp, float chit, float chi, float hx,
                                             float hy, float hz, float jpx, float jpy, float jpz) {
    Fcm27 c;
    c.chit = chit;
    c.chi = chi;
    const float r1 = 1.0f - kp.omD;
    c.v[0] = r1 * (jpx - chi * hx);
    c.v[1] = r1 * (jpy - chi * hy);
    c.v[2] = r1 * (jpz - chi * hz);
    const float u[3] = {hx, hy, hz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float uu = u[a] * u[a];
        c.W[a][0] = 1.0f / 6.0f; c.W[a][1] = 2.0f / 3.0f; c.W[a][2] = 1.0f / 6.0f;
        c.dE[a][1] = -uu;
        c.dE[a][0] = 0.5f * (uu - u[a]);
        c.dE[a][2] = 0.5f * (uu + u[a]);
        c.G[a][1] = -2.0f * u[a];
        c.G[a][0] = u[a] - 0.5f;
        c.G[a][2] = u[a] + 0.5f;
    }
    return c;
}
__device__ __forceinline__ float fcm27_value(const Fcm27& c, int i) {
    const int cx = cx27(i) + 1, cy = cy27(i) + 1, cz = cz27(i) + 1;
    const float Ex = c.W[0][cx] + c.dE[0][cx], Ey = c.W[1][cy] + c.dE[1][cy],
                Ez = c.W[2][cz] + c.dE[2][cz];
    // Ex Ey Ez - Wx Wy Wz without cancellation
    const float dprod = c.dE[0][cx] * Ey * Ez + c.W[0][cx] * c.dE[1][cy] * Ez +
                        c.W[0][cx] * c.W[1][cy] * c.dE[2][cz];
    const float vt = c.v[0] * c.G[0][cx] * Ey * Ez + c.v[1] * Ex * c.G[1][cy] * Ez +
                     c.v[2] * Ex * Ey * c.G[2][cz];
    return c.chit * w27(i) + c.chi * dprod + vt;
}

// First moments sum_i c_i (Phi_i - w_i) = sum_i c_i Phi_i of the D3Q27 scalar.
__device__ __forceinline__ void scalar_first_moments27(const float (&p)[27], float& jpx,
                                                       float& jpy, float& jpz) {
    jpx = 0.0f; jpy = 0.0f; jpz = 0.0f;
#pragma unroll
    for (int i = 1; i < 27; i += 2) {
        const float dm = p[i] - p[i + 1];
        if (cx27(i)) jpx += cx27(i) * dm;
        if (cy27(i)) jpy += cy27(i) * dm;
        if (cz27(i)) jpz += cz27(i) * dm;
    }
}

// D3Q27 factorized central moments (Eq. 37-51) with every rate of order >= 2
// equal to 1: the moments in the frame of u relax to their lattice
// equilibria chi (1, 0, 1/3)^(x) per axis, except the first-order ones,
// v = (1 - omega_D) (sum c Phi - chi u) with omega_D from Eq. 51.  The
// post-collision populations are therefore
//   chi Ex Ey Ez + vx Gx Ey Ez + vy Ex Gy Ez + vz Ex Ey Gz,
// E(0) = 2/3 - u^2, E(+-1) = (1/3 + u^2 +- u)/2 (moments (1, 0, 1/3)),
// G(0) = -2u, G(+-1) = (2u +- 1)/2 (moments (0, 1, 0)), both inverted in the
// frame of u.  Held as deviations: Phi* - w = (chi - 1) w + chi (Ex Ey Ez -
// w) + v-terms, with Ex Ey Ez - w expanded in the small parts dE = E - w1.
// p holds the pre-collision populations on entry (only the closing sum of
// the rest population reads them) and the post-collision ones on return;
// jp: their first moments, computed before.
__device__ __forceinline__ void collide_fcm27(const KParams& kp, float (&p)[27], float chit,
                                              float chi, float hx, float hy, float hz, float jpx,
                                              float jpy, float jpz) {
    const Fcm27 c = fcm27_setup(kp, chit, chi, hx, hy, hz, jpx, jpy, jpz);
    float psum = 0.0f;
#pragma unroll
    for (int i = 1; i < 27; ++i) {
        const float nv = fcm27_value(c, i);
        psum += nv - p[i];
        p[i] = nv;
    }
    // the rest population closes the sum (its reconstruction
    // chit w_0 + chi dprod_0 + vt_0 in exact arithmetic): sum Phi changes
    // only by the rounding of Phi_0, not by that of the 27-term chi
    p[0] -= psum;
}

// SL: scalar lattice, D3Q7 BGK or D3Q27 factorized central moments.
// SCALED (16-bit storage, D3Q7 scalar): f and p hold the storage units
// scale_f (f - w) and scale_phi (Phi - w); the scales are applied to the few
// moments and output coefficients instead of to every population.
template <int SL = 7, bool SCALED = false>
__device__ __forceinline__ void collide_cumulant(const KParams& kp, float (&f)[27],
                                                 float (&p)[ScalarLat<SL>::NS]) {
    static_assert(SL == 7 || SL == 27, "the cumulant model runs with the D3Q7 or D3Q27 scalar");
    static_assert(!(SCALED && SL == 27), "the D3Q27 scalar takes unscaled populations");
    constexpr int NS = ScalarLat<SL>::NS;
    float chs = 0.0f;  // chi - 1 in storage units (Phi is held as Phi - w)
#pragma unroll
    for (int k = 0; k < NS; ++k) chs += p[k];
    float chit, chi, hx, hy, hz;
    if constexpr (SL == 27) {
        float jpx, jpy, jpz;
        scalar_first_moments27(p, jpx, jpy, jpz);
        cumulant_fluid<SCALED>(kp, f, chs, chit, chi, hx, hy, hz);
        collide_fcm27(kp, p, chit, chi, hx, hy, hz, jpx, jpy, jpz);
    } else {
        cumulant_fluid<SCALED>(kp, f, chs, chit, chi, hx, hy, hz);
        // scalar (Eq. 28-30) with the half-force velocity and the molecular D;
        // non-equilibrium form whose parts sum to zero, so sum Phi is conserved
        // up to the rounding of the stored results (see collide_bgk)
        const float omp = kp.omp0;
        const float pe = w7(1) * chs, pa = (SCALED ? kp.sp : 1.0f) * w7(1) * 4.0f * chi;
        float nq[7];
        nq[1] = p[1] - (pe + pa * hx);
        nq[2] = p[2] - (pe - pa * hx);
        nq[3] = p[3] - (pe + pa * hy);
        nq[4] = p[4] - (pe - pa * hy);
        nq[5] = p[5] - (pe + pa * hz);
        nq[6] = p[6] - (pe - pa * hz);
        nq[0] = -(((nq[1] + nq[2]) + (nq[3] + nq[4])) + (nq[5] + nq[6]));
#pragma unroll
        for (int k = 0; k < 7; ++k) p[k] -= omp * nq[k];
    }
}

}  // namespace lbmgpu
