/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of one lock-exchange LBM time
 * step (Adekanye et al., "GPU accelerated LBM simulations of dilute gravity
 * currents", arXiv 2112.08479).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this code.  It shares no code, table,
 * header or constant generator with the CUDA library, and the CUDA library
 * never calls it.
 *
 * What it computes, per time step, at every node (lattice units, dx = dt = 1,
 * c_s^2 = 1/3 for the fluid):
 *   1. chi = sum_k Phi_k                                   (Sec. 2.3.1, Eq. 27)
 *   2. F = g' chi e^g                                      (Sec. 2.1,  Eq. 11)
 *   3. rho = sum_i f_i, rho u = sum_i c_i f_i + F/2        (Sec. 2.2,  Eq. 19-20)
 *   4. fluid collision, either
 *      BGK + Smagorinsky (Sec. 2.3.1, Eq. 21-26, 32-34), or
 *      cumulant (Sec. 2.3.1 "VirtualFluids", Eq. 54-58)
 *   5. scalar BGK collision on D3Q7 (Eq. 28-30, 35)
 *   6. streaming f_i(x + c_i, t + 1) = f*_i(x, t) (Eq. 17), written as a pull
 *      with half-way bounce-back at the x and z walls (Sec. 2.5) and periodic y.
 *
 * Layout: array of structures, node-major,
 *   f[((z*ny + y)*nx + x)*Q + i],   Phi[((z*ny + y)*nx + x)*NS + k],
 * NS = 7 (D3Q7), 6 (D3Q6) or 27 (D3Q27) scalar populations.
 * Two arrays, no in-place tricks, no blocking, no fusion beyond the above.
 *
 * Readings where the paper is silent or garbled (named R1..R17 in the design
 * notes; each is marked where it is used below):
 *   R1  D3Q7 scalar lattice, w0 = 1/4, w1..6 = 1/8, c_sPhi^2 = 1/4.
 *   R2  nu_T = (C_s Delta)^2 |S|, classical C_s, Delta = 1.
 *   R3  |S| = sqrt(2 S:S), S = -Pi / (2 rho c_s^2 tau_eff) gives the closed form
 *       tau_eff = (tau0 + sqrt(tau0^2 + 18 sqrt(2) C_s^2 q / rho)) / 2.
 *   R4  D_eff = D + nu_T / Sc_T.
 *   R5  Guo prefactor uses the local tau_eff.
 *   R6  compressible second-order equilibrium (Eq. 22).
 *   R7  cumulant: first order shifted by F/rho, second order relaxed with
 *       omega1 (shear, Eq. 58) and omega_bulk (trace), order >= 3 relaxed to 0
 *       with omega_high.
 *   R8  the force uses the pre-collision chi; the scalar equilibrium uses the
 *       same force-shifted u as the fluid.
 *   R9  walls on both x ends and both z ends, y periodic.
 *   R10 interface noise on column x0 - 1 from splitmix64(seed ^ n).
 *   R11 front = largest x whose span-averaged column maximum is >= threshold,
 *       linearly interpolated to the threshold crossing.
 *   R18 with periodic x ends the front is searched in x < (nx + x0) / 2.
 *   R12 F_w = sum over the bottom plane of nu (9 u_x(z=0) - u_x(z=1)) / 3.
 *
 * Parity pins: every function here is pinned by tests against closed forms,
 * invariants and brute force (moment identities, conservation, Poiseuille,
 * Taylor-Green, Gaussian diffusion, cumulant product identity, splitmix64
 * published vector).  The lock-exchange run as a whole has no closed form:
 * "parity unpinned" beyond those pins.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the node loops (collision, streaming, macroscopic fields).
 * Every node is computed on its own from the previous arrays, so the result
 * does not depend on the thread count; reductions (F_w, budgets, front)
 * stay serial.  1 unless orc_set_threads says otherwise. */
static int g_threads = 1;
int orc_set_threads(int n) {
#ifdef _OPENMP
    g_threads = n < 1 ? 1 : n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}
int orc_threads(void) { return g_threads; }

typedef struct {
    int nx, ny, nz;
    int model;          /* 0 = BGK-Smagorinsky D3Q19, 1 = cumulant D3Q27 */
    int periodic_x;     /* 0: half-way bounce-back walls at both x ends */
    int periodic_z;     /* 0: half-way bounce-back walls at both z ends */
    int no_collide;     /* 1: skip all collisions (pure streaming) */
    int pad_;
    double nu;          /* molecular viscosity */
    double D;           /* molecular scalar diffusivity */
    double cs_smag;     /* Smagorinsky constant (classical, R2) */
    double sc_t;        /* turbulent Schmidt number (R4) */
    double gprime;      /* reduced gravity g' (alpha g with rho_a = 1) */
    double eg[3];       /* unit vector of gravity, (0,0,-1) in the paper */
    double omega_bulk;  /* cumulant: rate of the second-order trace */
    double omega_high;  /* cumulant: rate of every cumulant of order >= 3 */
    int scalar;         /* scalar lattice: 0 D3Q7 BGK (R1), 1 D3Q6 BGK (Eq. 29-31),
                           2 D3Q27 factorized central moments (Eq. 37-51) */
    int pad2_;
    double omega_phi_high; /* D3Q27 scalar: rate of every factorized moment of
                              order >= 2 (Eq. 50) */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Velocity sets.                                                           */
/* D3Q19 in the order of Eq. 23, weights of Eq. 24.                         */
static const int C19[19][3] = {
    { 0, 0, 0},
    { 1, 0, 0}, {-1, 0, 0}, { 0, 1, 0}, { 0,-1, 0}, { 0, 0, 1}, { 0, 0,-1},
    { 1, 1, 0}, {-1,-1, 0}, { 1,-1, 0}, {-1, 1, 0},
    { 1, 0, 1}, {-1, 0,-1}, { 1, 0,-1}, {-1, 0, 1},
    { 0, 1, 1}, { 0,-1,-1}, { 0, 1,-1}, { 0,-1, 1}};

/* D3Q27: the 19 above, then the 8 corners (Eq. 36 prints only 7 of them;
 * the missing one is (1,-1,1)).  Corners are listed in opposite pairs.    */
static const int C27[27][3] = {
    { 0, 0, 0},
    { 1, 0, 0}, {-1, 0, 0}, { 0, 1, 0}, { 0,-1, 0}, { 0, 0, 1}, { 0, 0,-1},
    { 1, 1, 0}, {-1,-1, 0}, { 1,-1, 0}, {-1, 1, 0},
    { 1, 0, 1}, {-1, 0,-1}, { 1, 0,-1}, {-1, 0, 1},
    { 0, 1, 1}, { 0,-1,-1}, { 0, 1,-1}, { 0,-1, 1},
    { 1, 1, 1}, {-1,-1,-1}, { 1, 1,-1}, {-1,-1, 1},
    { 1,-1, 1}, {-1, 1,-1}, {-1, 1, 1}, { 1,-1,-1}};

/* D3Q7 scalar lattice (R1): rest, then +-x, +-y, +-z. */
static const int C7[7][3] = {
    { 0, 0, 0}, { 1, 0, 0}, {-1, 0, 0}, { 0, 1, 0}, { 0,-1, 0}, { 0, 0, 1}, { 0, 0,-1}};

/* D3Q6 scalar lattice in the order of Eq. 31, w = 1/6 (Sec. 2.3.1). */
static const int C6[6][3] = {
    { 1, 0, 0}, {-1, 0, 0}, { 0, 1, 0}, { 0,-1, 0}, { 0, 0, 1}, { 0, 0,-1}};

static int nsq(const int c[3]) { return c[0]*c[0] + c[1]*c[1] + c[2]*c[2]; }

/* Eq. 24 */
static double w19(int i) {
    int n = nsq(C19[i]);
    return n == 0 ? 1.0/3.0 : (n == 1 ? 1.0/18.0 : 1.0/36.0);
}
/* D3Q27 weights: tensor product of (1/6, 2/3, 1/6) per axis. */
static double w27(int i) {
    double w = 1.0;
    for (int a = 0; a < 3; ++a) w *= (C27[i][a] == 0) ? 2.0/3.0 : 1.0/6.0;
    return w;
}
/* R1 */
static double w7(int k) { return k == 0 ? 0.25 : 0.125; }

static int nq(const orc_params* p) { return p->model == 1 ? 27 : 19; }
static int ns(const orc_params* p) { return p->scalar == 1 ? 6 : (p->scalar == 2 ? 27 : 7); }
static const int (*sset(const orc_params* p))[3] {
    return p->scalar == 1 ? C6 : (p->scalar == 2 ? C27 : C7);
}
static double wsc(const orc_params* p, int k) {
    return p->scalar == 1 ? 1.0/6.0 : (p->scalar == 2 ? w27(k) : w7(k));
}
static const int (*cset(const orc_params* p))[3] { return p->model == 1 ? C27 : C19; }
static double wq(const orc_params* p, int i) { return p->model == 1 ? w27(i) : w19(i); }

/* index of the direction opposite to c_i, found by search */
static int opposite(const int (*c)[3], int q, int i) {
    for (int j = 0; j < q; ++j)
        if (c[j][0] == -c[i][0] && c[j][1] == -c[i][1] && c[j][2] == -c[i][2]) return j;
    return -1;
}

/* exported views of the tables, so tests can check them against the paper */
int orc_q(int model) { return model == 1 ? 27 : 19; }
void orc_velocities(int model, int* c_out, double* w_out) {
    orc_params p; memset(&p, 0, sizeof p); p.model = model;
    int q = nq(&p);
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) c_out[3*i + a] = cset(&p)[i][a];
        w_out[i] = wq(&p, i);
    }
}
void orc_velocities_q7(int* c_out, double* w_out) {
    for (int k = 0; k < 7; ++k) {
        for (int a = 0; a < 3; ++a) c_out[3*k + a] = C7[k][a];
        w_out[k] = w7(k);
    }
}
int orc_ns(int scalar) { return scalar == 1 ? 6 : (scalar == 2 ? 27 : 7); }
void orc_velocities_scalar(int scalar, int* c_out, double* w_out) {
    orc_params p; memset(&p, 0, sizeof p); p.scalar = scalar;
    for (int k = 0; k < ns(&p); ++k) {
        for (int a = 0; a < 3; ++a) c_out[3*k + a] = sset(&p)[k][a];
        w_out[k] = wsc(&p, k);
    }
}

/* ------------------------------------------------------------------------ */
/* Equilibria.                                                              */

/* Eq. 22 with c_s^2 = 1/3 (R6). */
void orc_feq_q19(double rho, const double u[3], double* feq) {
    double uu = u[0]*u[0] + u[1]*u[1] + u[2]*u[2];
    for (int i = 0; i < 19; ++i) {
        double cu = C19[i][0]*u[0] + C19[i][1]*u[1] + C19[i][2]*u[2];
        feq[i] = w19(i) * rho * (1.0 + 3.0*cu + 4.5*cu*cu - 1.5*uu);
    }
}

/* Eq. 29 on D3Q7 with c_sPhi^2 = 1/4 (R1). */
void orc_phieq_q7(double chi, const double u[3], double* phieq) {
    for (int k = 0; k < 7; ++k) {
        double cu = C7[k][0]*u[0] + C7[k][1]*u[1] + C7[k][2]*u[2];
        phieq[k] = w7(k) * chi * (1.0 + 4.0*cu);
    }
}

/* ------------------------------------------------------------------------ */
/* Smagorinsky closure (Eq. 32-34, reading R3).                            */
double orc_tau_eff(double tau0, double cs_smag, double q, double rho) {
    return 0.5 * (tau0 + sqrt(tau0*tau0 + 18.0*sqrt(2.0)*cs_smag*cs_smag*q/rho));
}

/* ------------------------------------------------------------------------ */
/* Macroscopic moments with the half-force shift (Eq. 19-20, 27, 11).      */
static void node_moments(const orc_params* p, const double* f, const double* phi,
                         double* rho, double u[3], double* chi, double F[3]) {
    int q = nq(p);
    const int (*c)[3] = cset(p);
    double x = 0.0;
    for (int k = 0; k < ns(p); ++k) x += phi[k];
    *chi = x;
    for (int a = 0; a < 3; ++a) F[a] = p->gprime * x * p->eg[a];
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < q; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) j[a] += c[i][a] * f[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5*F[a]) / r;
}

/* ------------------------------------------------------------------------ */
/* BGK-Smagorinsky collision with the Guo source (Eq. 21-26, 32-34).       */
static void collide_bgk(const orc_params* p, const double* f, double rho,
                        const double u[3], const double F[3],
                        double* fo, double* nu_t) {
    double feq[19];
    orc_feq_q19(rho, u, feq);
    /* Pi_ab = sum_i c_ia c_ib (f_i - feq_i)  (the tensor of Eq. 33) */
    double Pi[3][3] = {{0}};
    for (int i = 0; i < 19; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                Pi[a][b] += C19[i][a] * C19[i][b] * (f[i] - feq[i]);
    double qq = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) qq += Pi[a][b] * Pi[a][b];
    double q = sqrt(qq);
    double tau0 = 3.0 * p->nu + 0.5;                       /* Eq. 25 */
    double tau = orc_tau_eff(tau0, p->cs_smag, q, rho);    /* R3 */
    *nu_t = (tau - tau0) / 3.0;
    for (int i = 0; i < 19; ++i) {
        const int* ci = C19[i];
        double cu = ci[0]*u[0] + ci[1]*u[1] + ci[2]*u[2];
        /* Eq. 26: w [ (c - u)/c_s^2 + (c.u) c / c_s^4 ] . F, prefactor (1 - 1/2tau) */
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            s += (3.0*(ci[a] - u[a]) + 9.0*cu*ci[a]) * F[a];
        double S = (1.0 - 0.5/tau) * w19(i) * s;
        fo[i] = f[i] - (f[i] - feq[i]) / tau + S;          /* Eq. 17, 21 */
    }
}

/* ------------------------------------------------------------------------ */
/* Cumulant collision (Eq. 54-58, reading R7).                             */
/* The moment generating function G(Xi) = sum_i f_i exp(Xi . c_i) is held   */
/* by its Taylor coefficients g[a][b][c] of Xi^a Y^b Z^c with a, b, c <= 2,  */
/* i.e. in the ring R[Xi,Y,Z]/(Xi^3, Y^3, Z^3).  The quotient map is a ring  */
/* homomorphism, so ln and exp computed in it give exactly the coefficients  */
/* with a, b, c <= 2 of the full series; total degree <= 6 makes the series  */
/* of ln(1 + H) and exp(K) finite when H, K have no constant term.          */
typedef double ring[3][3][3];

static void ring_mul(const ring A, const ring B, ring out) {
    ring t;
    memset(t, 0, sizeof t);
    for (int a1 = 0; a1 < 3; ++a1) for (int b1 = 0; b1 < 3; ++b1) for (int c1 = 0; c1 < 3; ++c1)
    for (int a2 = 0; a1 + a2 < 3; ++a2) for (int b2 = 0; b1 + b2 < 3; ++b2) for (int c2 = 0; c1 + c2 < 3; ++c2)
        t[a1+a2][b1+b2][c1+c2] += A[a1][b1][c1] * B[a2][b2][c2];
    memcpy(out, t, sizeof t);
}

static const double FACT[3] = {1.0, 1.0, 2.0};

/* ln(1 + H) for H with zero constant term: sum_{k=1..6} (-1)^(k+1) H^k / k */
static void ring_log1p(const ring H, ring out) {
    ring P, S;
    memcpy(P, H, sizeof P);
    memcpy(S, H, sizeof S);
    for (int k = 2; k <= 6; ++k) {
        ring_mul(P, H, P);
        double s = ((k % 2) ? 1.0 : -1.0) / k;
        for (int a = 0; a < 27; ++a) (&S[0][0][0])[a] += s * (&P[0][0][0])[a];
    }
    memcpy(out, S, sizeof S);
}

/* exp(K) for K with zero constant term: sum_{k=0..6} K^k / k! */
static void ring_exp(const ring K, ring out) {
    ring P, S;
    memset(S, 0, sizeof S);
    S[0][0][0] = 1.0;
    memcpy(P, K, sizeof P);
    double fk = 1.0;
    for (int k = 1; k <= 6; ++k) {
        if (k > 1) ring_mul(P, K, P);
        fk *= k;
        for (int a = 0; a < 27; ++a) (&S[0][0][0])[a] += (&P[0][0][0])[a] / fk;
    }
    memcpy(out, S, sizeof S);
}

/* raw moments m_abc = sum_i cx^a cy^b cz^c f_i (Eq. 18), a, b, c <= 2 */
static void raw_moments27(const double* f, ring m) {
    memset(m, 0, sizeof(ring));
    for (int i = 0; i < 27; ++i)
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c) {
            double v = f[i];
            for (int k = 0; k < a; ++k) v *= C27[i][0];
            for (int k = 0; k < b; ++k) v *= C27[i][1];
            for (int k = 0; k < c; ++k) v *= C27[i][2];
            m[a][b][c] += v;
        }
}

/* inverse of the per-axis Vandermonde map {f(-1), f(0), f(1)} -> {m0, m1, m2}:
 * f(0) = m0 - m2, f(+-1) = (m2 +- m1) / 2, applied on all three axes */
static void f_from_moments27(const ring m, double* f) {
    for (int i = 0; i < 27; ++i) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c) {
            int idx[3] = {a, b, c};
            double v = m[a][b][c];
            for (int d = 0; d < 3; ++d) {
                int cv = C27[i][d], n = idx[d];
                double coef;
                if (cv == 0) coef = (n == 0) ? 1.0 : (n == 2 ? -1.0 : 0.0);
                else coef = (n == 0) ? 0.0 : (n == 1 ? 0.5*cv : 0.5);
                v *= coef;
            }
            s += v;
        }
        f[i] = s;
    }
}

/* Cumulants C_abc = a! b! c! [Xi^a Y^b Z^c] ln G  (Eq. 54), a, b, c <= 2.
 * C[0] holds ln rho.  Output index (a*3 + b)*3 + c. */
void orc_cumulants27(const double* f, double* Cout) {
    ring m, g, H, L;
    raw_moments27(f, m);
    double rho = m[0][0][0];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c)
        g[a][b][c] = m[a][b][c] / (FACT[a]*FACT[b]*FACT[c]);
    for (int a = 0; a < 27; ++a) (&H[0][0][0])[a] = (&g[0][0][0])[a] / rho;
    H[0][0][0] = 0.0;                      /* G / rho = 1 + H */
    ring_log1p(H, L);
    L[0][0][0] = log(rho);
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c)
        Cout[(a*3 + b)*3 + c] = L[a][b][c] * FACT[a]*FACT[b]*FACT[c];
}

/* Inverse of orc_cumulants27: distributions whose cumulants are C. */
void orc_f_from_cumulants27(const double* Cin, double* f) {
    ring K, E, m;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c)
        K[a][b][c] = Cin[(a*3 + b)*3 + c] / (FACT[a]*FACT[b]*FACT[c]);
    double rho = exp(K[0][0][0]);
    K[0][0][0] = 0.0;
    ring_exp(K, E);
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c)
        m[a][b][c] = rho * E[a][b][c] * FACT[a]*FACT[b]*FACT[c];
    f_from_moments27(m, f);
}

#define CI(a, b, c) (((a)*3 + (b))*3 + (c))

static void collide_cumulant(const orc_params* p, const double* f, double rho,
                             const double F[3], double* fo) {
    double C[27];
    orc_cumulants27(f, C);
    double om1 = 1.0 / (3.0*p->nu + 0.5);          /* Eq. 58 */
    double om2 = p->omega_bulk, omh = p->omega_high;
    double Cs[27];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c) {
        int n = a + b + c, id = CI(a, b, c);
        if (n == 0) Cs[id] = C[id];                   /* Eq. 56: rho conserved */
        else if (n >= 3) Cs[id] = (1.0 - omh) * C[id];/* Eq. 55, C^eq = 0 */
        else Cs[id] = 0.0;                            /* filled below */
    }
    /* first order (Eq. 57): conserved momentum plus the body-force impulse */
    double j[3] = {C[CI(1,0,0)]*rho, C[CI(0,1,0)]*rho, C[CI(0,0,1)]*rho};
    Cs[CI(1,0,0)] = (j[0] + F[0]) / rho;
    Cs[CI(0,1,0)] = (j[1] + F[1]) / rho;
    Cs[CI(0,0,1)] = (j[2] + F[2]) / rho;
    /* second order (Eq. 55 with omega1 from Eq. 58): shear parts with omega1,
     * the trace with omega_bulk towards its equilibrium 3 c_s^2 = 1 */
    Cs[CI(1,1,0)] = (1.0 - om1) * C[CI(1,1,0)];
    Cs[CI(1,0,1)] = (1.0 - om1) * C[CI(1,0,1)];
    Cs[CI(0,1,1)] = (1.0 - om1) * C[CI(0,1,1)];
    double cxx = C[CI(2,0,0)], cyy = C[CI(0,2,0)], czz = C[CI(0,0,2)];
    double d1 = (1.0 - om1) * (cxx - cyy);
    double d2 = (1.0 - om1) * (cxx - czz);
    double tr = (1.0 - om2) * (cxx + cyy + czz) + om2 * 1.0;
    double nxx = (tr + d1 + d2) / 3.0;
    Cs[CI(2,0,0)] = nxx;
    Cs[CI(0,2,0)] = nxx - d1;
    Cs[CI(0,0,2)] = nxx - d2;
    orc_f_from_cumulants27(Cs, fo);
}

/* ------------------------------------------------------------------------ */
/* Scalar collisions.                                                       */

/* Eq. 29 on D3Q6, literal: c_s^2 = 1/3, w = 1/6. */
void orc_phieq_q6(double chi, const double u[3], double* phieq) {
    for (int k = 0; k < 6; ++k) {
        double cu = C6[k][0]*u[0] + C6[k][1]*u[1] + C6[k][2]*u[2];
        phieq[k] = chi * (1.0 + 3.0*cu) / 6.0;
    }
}

/* D3Q27 factorized central moments (Eq. 37-51).  Central moments of Phi in
 * the frame moving with u (Eq. 39), factorized moments M (Eq. 40-49), which
 * subtract from kappa_abc the lattice equilibrium share (1/3)^m kappa_a'b'c',
 * m the number of indices equal to 2 and a'b'c' the indices with every 2
 * replaced by 0 (Eq. 46 is garbled in the text: the same rule gives
 * kappa_220 - kappa_000 / 9).  M_000 = chi is conserved, the first-order M
 * relax with omega from D = (1/omega - 1/2) / 3 (Eq. 51), all others with
 * omega_phi_high towards 0 (Eq. 50).  Back: kappa = M + (1/3)^m M_a'b'c', raw
 * moments by the binomial frame shift, populations by the per-axis inverse
 * Vandermonde map. */
static void collide_fcm27(const orc_params* p, const double* phi, const double u[3],
                          double Deff, double* phio) {
    ring K, M, Ks, m;
    memset(K, 0, sizeof K);
    for (int i = 0; i < 27; ++i)
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c) {
            double v = phi[i];
            for (int k = 0; k < a; ++k) v *= (C27[i][0] - u[0]);
            for (int k = 0; k < b; ++k) v *= (C27[i][1] - u[1]);
            for (int k = 0; k < c; ++k) v *= (C27[i][2] - u[2]);
            K[a][b][c] += v;
        }
    double third[4] = {1.0, 1.0/3.0, 1.0/9.0, 1.0/27.0};
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c) {
        int m2 = (a == 2) + (b == 2) + (c == 2);
        M[a][b][c] = K[a][b][c] - (m2 ? third[m2] * K[a % 2][b % 2][c % 2] : 0.0);
    }
    double omD = 1.0 / (3.0*Deff + 0.5);
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c) {
        int n = a + b + c;
        if (n == 1) M[a][b][c] *= (1.0 - omD);
        else if (n >= 2) M[a][b][c] *= (1.0 - p->omega_phi_high);
    }
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c) {
        int m2 = (a == 2) + (b == 2) + (c == 2);
        Ks[a][b][c] = M[a][b][c] + (m2 ? third[m2] * M[a % 2][b % 2][c % 2] : 0.0);
    }
    /* raw moments m_abc = sum_{a'<=a,...} C(a,a') u^(a-a') ... kappa_a'b'c' */
    static const double BIN[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};
    memset(m, 0, sizeof m);
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c)
    for (int a1 = 0; a1 <= a; ++a1) for (int b1 = 0; b1 <= b; ++b1) for (int c1 = 0; c1 <= c; ++c1)
        m[a][b][c] += BIN[a][a1] * pow(u[0], a - a1) * BIN[b][b1] * pow(u[1], b - b1)
                    * BIN[c][c1] * pow(u[2], c - c1) * Ks[a1][b1][c1];
    f_from_moments27(m, phio);
}

/* Scalar collision on the lattice p->scalar (Eq. 28-30, 35 with readings R1,
 * R4; Eq. 37-51 for D3Q27). */
static void collide_scalar(const orc_params* p, const double* phi, double chi,
                           const double u[3], double nu_t, double* phio) {
    double Deff = p->D + (p->model == 0 ? nu_t / p->sc_t : 0.0);
    if (p->scalar == 2) { collide_fcm27(p, phi, u, Deff, phio); return; }
    double phieq[7];
    double tauphi;
    if (p->scalar == 1) {
        tauphi = 0.5 + 3.0 * Deff;                     /* D = c_s^2 (tau - 1/2), c_s^2 = 1/3 */
        orc_phieq_q6(chi, u, phieq);
    } else {
        tauphi = 0.5 + 4.0 * Deff;                     /* c_sPhi^2 = 1/4 on D3Q7 */
        orc_phieq_q7(chi, u, phieq);
    }
    for (int k = 0; k < ns(p); ++k) phio[k] = phi[k] - (phi[k] - phieq[k]) / tauphi;
}

/* One node: fluid + scalar collision.  Exported for the single-node pins. */
void orc_collide_node(const orc_params* p, const double* f, const double* phi,
                      double* fo, double* phio) {
    int q = nq(p);
    if (p->no_collide) {
        memcpy(fo, f, sizeof(double)*q);
        memcpy(phio, phi, sizeof(double)*ns(p));
        return;
    }
    double rho, u[3], chi, F[3], nu_t = 0.0;
    node_moments(p, f, phi, &rho, u, &chi, F);
    if (p->model == 0) collide_bgk(p, f, rho, u, F, fo, &nu_t);
    else collide_cumulant(p, f, rho, F, fo);
    collide_scalar(p, phi, chi, u, nu_t, phio);
}

/* Eddy viscosity nu_T = (tau_eff - tau0) / 3 that the BGK collision uses at
 * one node (Eq. 32-34, reading R3).  Exported for the closure pins. */
double orc_bgk_nu_t(const orc_params* p, const double* f, const double* phi) {
    double rho, u[3], chi, F[3], fo[19], nu_t = 0.0;
    node_moments(p, f, phi, &rho, u, &chi, F);
    collide_bgk(p, f, rho, u, F, fo, &nu_t);
    return nu_t;
}

/* ------------------------------------------------------------------------ */
/* Streaming (Eq. 17) as a pull with half-way bounce-back (Sec. 2.5).      */
static long node_index(const orc_params* p, int x, int y, int z) {
    return ((long)z * p->ny + y) * p->nx + x;
}

/* upwind neighbour x - c: returns 0 when it lies outside a wall */
static int upwind(const orc_params* p, int x, int y, int z, const int c[3], long* src) {
    int xs = x - c[0], ys = y - c[1], zs = z - c[2];
    ys = ((ys % p->ny) + p->ny) % p->ny;
    if (xs < 0 || xs >= p->nx) {
        if (!p->periodic_x) return 0;
        xs = ((xs % p->nx) + p->nx) % p->nx;
    }
    if (zs < 0 || zs >= p->nz) {
        if (!p->periodic_z) return 0;
        zs = ((zs % p->nz) + p->nz) % p->nz;
    }
    *src = node_index(p, xs, ys, zs);
    return 1;
}

/* post-collision arrays -> streamed arrays */
void orc_stream(const orc_params* p, const double* fpost, const double* phipost,
                double* f, double* phi) {
    int q = nq(p);
    const int (*c)[3] = cset(p);
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
    for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
        long n = node_index(p, x, y, z), s;
        for (int i = 0; i < q; ++i) {
            if (upwind(p, x, y, z, c[i], &s)) f[n*q + i] = fpost[s*q + i];
            else f[n*q + i] = fpost[n*q + opposite(c, q, i)];
        }
        const int S = ns(p);
        const int (*cs)[3] = sset(p);
        for (int k = 0; k < S; ++k) {
            if (upwind(p, x, y, z, cs[k], &s)) phi[n*S + k] = phipost[s*S + k];
            else phi[n*S + k] = phipost[n*S + opposite(cs, S, k)];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Diagnostics (Sec. 3.1 and 3.2, Eq. 62-64; readings R11, R12).           */

/* rho, u (with the half-force shift) and chi of every node. u is node-major
 * [n*3 + a]. */
void orc_macros(const orc_params* p, const double* f, const double* phi,
                double* rho, double* u, double* chi) {
    int q = nq(p);
    long N = (long)p->nx * p->ny * p->nz;
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
    for (long n = 0; n < N; ++n) {
        double r, uu[3], x, F[3];
        node_moments(p, f + n*q, phi + n*ns(p), &r, uu, &x, F);
        if (rho) rho[n] = r;
        if (u) for (int a = 0; a < 3; ++a) u[n*3 + a] = uu[a];
        if (chi) chi[n] = x;
    }
}

/* F_w = sum_{x,y} tau_w, tau_w = nu * du/dz at the wall (Eq. 62, 64), where
 * du/dz is the derivative at z = -1/2 of the quadratic through u = 0 at the
 * wall and the first two nodes, i.e. (9 u(0) - u(1)) / 3. */
double orc_wall_friction(int nx, int ny, int nz, double nu, const double* u) {
    double s = 0.0;
    if (nz < 2) return 0.0;
    for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
        long n0 = ((long)0*ny + y)*nx + x, n1 = ((long)1*ny + y)*nx + x;
        s += nu * (9.0*u[n0*3 + 0] - u[n1*3 + 0]) / 3.0;
    }
    return s;
}

/* Front (Sec. 3.1): chibar(x,z) = mean_y chi, m(x) = max_z chibar, x_f = the
 * largest x < xlim with m(x) >= thr, moved to the linear threshold crossing
 * between x_f and x_f + 1 unless x_f = xlim - 1.  xlim = nx with walls at the
 * x ends; with periodic ends (Fig. 4b) the columns ahead of the lock,
 * xlim = (nx + x0) / 2 (orc_front_xlim).  Returns the node coordinate (-1
 * when no column reaches thr). */
int orc_front_xlim(int nx, int x0, int periodic_x) {
    if (!periodic_x) return nx;
    int h = (nx + x0) / 2;
    return h < 1 ? 1 : h;
}

double orc_front_node_lim(int nx, int ny, int nz, const double* chi, double thr, int xlim) {
    double* m = (double*)malloc(sizeof(double) * nx);
    for (int x = 0; x < nx; ++x) m[x] = -INFINITY;
    for (int z = 0; z < nz; ++z)
    for (int x = 0; x < nx; ++x) {
        double s = 0.0;
        for (int y = 0; y < ny; ++y) s += chi[((long)z*ny + y)*nx + x];
        s /= ny;
        if (s > m[x]) m[x] = s;
    }
    int xf = -1;
    for (int x = xlim - 1; x >= 0; --x) if (m[x] >= thr) { xf = x; break; }
    double r;
    if (xf < 0) r = -1.0;
    else if (xf == xlim - 1) r = (double)xf;
    else r = xf + (m[xf] - thr) / (m[xf] - m[xf + 1]);
    free(m);
    return r;
}

double orc_front_node(int nx, int ny, int nz, const double* chi, double thr) {
    return orc_front_node_lim(nx, ny, nz, chi, thr, nx);
}

/* out[0] = front position (x_f + 1/2 - x0) / H, out[1] = F_w,
 * out[2] = sum (rho - 1), out[3] = sum chi, out[4] = front node coordinate */
void orc_diag(const orc_params* p, const double* f, const double* phi,
              int x0, double H, double thr, double* out) {
    long N = (long)p->nx * p->ny * p->nz;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* u = (double*)malloc(sizeof(double) * N * 3);
    double* chi = (double*)malloc(sizeof(double) * N);
    orc_macros(p, f, phi, rho, u, chi);
    double xf = orc_front_node_lim(p->nx, p->ny, p->nz, chi, thr,
                                   orc_front_xlim(p->nx, x0, p->periodic_x));
    out[0] = (xf + 0.5 - x0) / H;
    out[1] = orc_wall_friction(p->nx, p->ny, p->nz, p->nu, u);
    double sm = 0.0, sc = 0.0;
    for (long n = 0; n < N; ++n) { sm += rho[n] - 1.0; sc += chi[n]; }
    out[2] = sm;
    out[3] = sc;
    out[4] = xf;
    free(rho); free(u); free(chi);
}

/* ------------------------------------------------------------------------ */
/* Time stepping.                                                           */

/* one step: collide at every node, then stream (Eq. 17) */
void orc_step(const orc_params* p, double* f, double* phi) {
    int q = nq(p);
    long N = (long)p->nx * p->ny * p->nz;
    double* fpost = (double*)malloc(sizeof(double) * N * q);
    const int S = ns(p);
    double* phipost = (double*)malloc(sizeof(double) * N * S);
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
    for (long n = 0; n < N; ++n)
        orc_collide_node(p, f + n*q, phi + n*S, fpost + n*q, phipost + n*S);
    orc_stream(p, fpost, phipost, f, phi);
    free(fpost); free(phipost);
}

/* nsteps steps in place; fw[n] (if given) receives F_w after step n + 1 */
void orc_run(const orc_params* p, int nsteps, double* f, double* phi, double* fw) {
    long N = (long)p->nx * p->ny * p->nz;
    double* u = fw ? (double*)malloc(sizeof(double) * N * 3) : NULL;
    for (int s = 0; s < nsteps; ++s) {
        orc_step(p, f, phi);
        if (fw) {
            orc_macros(p, f, phi, NULL, u, NULL);
            fw[s] = orc_wall_friction(p->nx, p->ny, p->nz, p->nu, u);
        }
    }
    free(u);
}

/* ------------------------------------------------------------------------ */
/* Initial condition (Sec. 2.5, Table 1; reading R10).                     */

/* splitmix64 output for state s (Steele, Lea & Flood 2014, as published by
 * Vigna): z = s + 0x9e3779b97f4a7c15, two xor-shift-multiply rounds. */
uint64_t orc_splitmix64(uint64_t s) {
    uint64_t z = s + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* chi0 = 1 for x < x0 else 0; column x0 - 1 gets amp * (2r - 1) with
 * r = (splitmix64(seed ^ n) >> 11) * 2^-53, n the linear node index */
void orc_lock_chi0(int nx, int ny, int nz, int x0, double amp, uint64_t seed, double* chi0) {
    for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
        long n = ((long)z*ny + y)*nx + x;
        double v = x < x0 ? 1.0 : 0.0;
        if (x == x0 - 1) {
            double r = (double)(orc_splitmix64(seed ^ (uint64_t)n) >> 11) * 0x1.0p-53;
            v += amp * (2.0*r - 1.0);
        }
        chi0[n] = v;
    }
}

/* rest state f_i = w_i (rho = 1, u = 0), Phi_k = w_k chi0 (the scalar
 * lattice's weights; for D3Q27 that is the moment equilibrium at u = 0) */
void orc_init(const orc_params* p, const double* chi0, double* f, double* phi) {
    int q = nq(p);
    long N = (long)p->nx * p->ny * p->nz;
    for (long n = 0; n < N; ++n) {
        for (int i = 0; i < q; ++i) f[n*q + i] = wq(p, i);
        for (int k = 0; k < ns(p); ++k) phi[n*ns(p) + k] = wsc(p, k) * chi0[n];
    }
}
