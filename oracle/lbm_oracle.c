/*
 * lbm_oracle.c -- plain FP64 CPU oracle for one time step of the two-component
 * colour-gradient lattice Boltzmann (LB) method on the D3Q19 lattice, as used in
 * Succi et al., "Towards Exascale Design of Soft Mesoscale Materials"
 * (arXiv:2005.12764).
 *
 * TEST INFRASTRUCTURE. This file is the slow, obviously-correct reference that the
 * GPU library is checked against. Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it. It shares no code, header, table
 * or constant generator with the GPU path.
 *
 * Every routine follows one passage of the paper (cited in its comment) or, where
 * the paper is silent, the published colour-gradient method it cites
 * (montessori2019mesoscale) in the reading stated beside the routine. Each phase
 * of a step is its own loop over all nodes, in the order of the method:
 *
 *   1. pull streaming with halfway bounce-back walls        Eq. (1), streaming text;
 *      optionally sliding y-walls                           sheared-bijel section
 *   2. moments rho_r, rho_b, j, phi                          Eq. (3)
 *   3. isotropic colour gradient                             stencil form of Eq. (10)
 *   4. forces: body + Kolmogorov + near-contact              Eq. (11); the film
 *      thickness of the near-contact force is measured on the previous step's
 *      colour field
 *   5. BGK collision of the total population + EDM source    Eqs. (1), (2), (5)-(9)
 *   6. colour-gradient perturbation (surface tension)        reading: generalised
 *                                                            perturbation operator
 *   7. recolouring of the two species                        reading: Latva-Kokko &
 *                                                            Rothman segregation
 *
 * or, with model = 1, the Shan-Chen binary mixture of the same section: phases 3-7
 * replaced by the cohesive force of Eq. (12) and a per-species BGK + EDM collision
 * (Eqs. (5)-(9)); the near-contact force is not part of that model.
 *
 * The only parallelism is an OpenMP "parallel for" over z-planes inside each phase;
 * each node is computed independently, so results do not depend on thread count.
 * Compile without fast-math and with -ffp-contract=off so x86 and Arm agree.
 *
 * Parity status: every routine here is pinned by a closed form, an invariant, a
 * special case or a brute-force check in tests/test_oracle_*.py, except the
 * near-contact force routine, whose exact numbers the paper does not fix
 * ("parity unpinned": it is pinned only qualitatively -- merging vs. no merging
 * in the sense of the capillary number N_c -- and by exact momentum balance).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* D3Q19 velocity set (Sec. "Basics of Lattice Boltzmann Method", Fig. 1).
 * The paper shows the set only as a figure; the standard set is one rest
 * velocity, the 6 face neighbours and the 12 edge neighbours of a cube.       */
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static double W[Q];   /* weights: 1/3 rest, 1/18 face, 1/36 edge (normalised to 1) */
static int OPP[Q];    /* index of -c_i                                              */
static double BPERT[Q];
static const double CS2 = 1.0 / 3.0; /* lattice speed of sound squared */
static int lattice_ready = 0;

static void lattice_init(void) {
    if (lattice_ready) return;
    for (int i = 0; i < Q; ++i) {
        int c2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
        W[i] = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
        /* Perturbation-operator constants B_i (reading, see or_perturb). */
        BPERT[i] = (c2 == 0) ? -2.0 / 9.0 : (c2 == 1) ? 1.0 / 54.0 : 1.0 / 27.0;
        OPP[i] = -1;
        for (int k = 0; k < Q; ++k)
            if (CX[k] == -CX[i] && CY[k] == -CY[i] && CZ[k] == -CZ[i]) OPP[i] = k;
    }
    lattice_ready = 1;
}

/* Export of the lattice tables (for the lattice pins). */
void or_lattice(int* c /* [Q][3] */, double* w, int* opp, double* bpert) {
    lattice_init();
    for (int i = 0; i < Q; ++i) {
        c[3 * i + 0] = CX[i];
        c[3 * i + 1] = CY[i];
        c[3 * i + 2] = CZ[i];
        w[i] = W[i];
        opp[i] = OPP[i];
        bpert[i] = BPERT[i];
    }
}

/* ------------------------------------------------------------------------- */
/* Parameters and state.                                                      */
typedef struct {
    int nx, ny, nz;        /* lattice size, x fastest                                */
    int wall_y, wall_z;    /* 1 = halfway bounce-back walls at both extremes         */
    double tau_r, tau_b;   /* relaxation times, nu_k = c_s^2 (tau_k - 1/2), Eq. (4)   */
    double sigma, beta;    /* surface tension, recolouring segregation parameter     */
    double A_nc, h_min, h_cut; /* near-contact amplitude A, plateau length, cutoff   */
    double g[3];           /* uniform body-force density                              */
    double kolmogorov_amp; /* F_x(y) = amp * sin(2 pi y / ny)                         */
    int nc_lag;            /* 1: near-contact ray reads phi of the previous step      */
    double wall_u;         /* sliding y-walls: the wall at y = ny - 1/2 moves with
                              (+wall_u, 0, 0), the one at y = -1/2 with (-wall_u, 0, 0) */
    int model;             /* 0: colour gradient; 1: Shan-Chen (Eqs. (5)-(9), (12))   */
    double G_sc;           /* Shan-Chen coupling G_C (> 0 repulsive)                 */
} or_params;

typedef struct {
    or_params p;
    long N;
    double *fr, *fb;   /* state: post-collision populations f*_i^k, layout [i][N] */
    double *gr, *gb;   /* post-stream populations of the current step            */
    double *rho_r, *rho_b, *jx, *jy, *jz, *phi, *phi_lag;
    double *Gx, *Gy, *Gz, *Fx, *Fy, *Fz;
    unsigned char* pin; /* pinning-site mask (1 = pin) or NULL                   */
    long steps;
} or_state;

static inline long nidx(const or_params* p, long x, long y, long z) {
    return (z * p->ny + y) * p->nx + x;
}
static inline long wrap(long a, long n) {
    a %= n;
    return a < 0 ? a + n : a;
}

/* ------------------------------------------------------------------------- */
/* Eq. (2): second-order equilibrium f_i^eq = w_i rho (1 + u.c_i/c_s^2 +
 * (c_ia c_ib - c_s^2 delta_ab) u_a u_b / (2 c_s^4)).                           */
void or_feq(double rho, const double u[3], double feq[Q]) {
    lattice_init();
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
        double qi = (cu * cu - CS2 * usq) / (2.0 * CS2 * CS2);
        feq[i] = W[i] * rho * (1.0 + cu / CS2 + qi);
    }
}

/* Eq. (9): exact-difference-method source, the difference of two equilibria,
 * S_i = f_i^eq(rho, u + F dt / rho) - f_i^eq(rho, u), with dt = 1.             */
void or_edm_source(double rho, const double u[3], const double F[3], double S[Q]) {
    double us[3] = {u[0] + F[0] / rho, u[1] + F[1] / rho, u[2] + F[2] / rho};
    double a[Q], b[Q];
    or_feq(rho, us, a);
    or_feq(rho, u, b);
    for (int i = 0; i < Q; ++i) S[i] = a[i] - b[i];
}

/* Eqs. (4), (7), (8): effective relaxation rate of the mixture. The viscosity of
 * each species is nu_k = c_s^2 (tau_k - 1/2); the mixture viscosity is the
 * density-weighted harmonic mean 1/nu = sum_k (rho_k/rho) / nu_k. Eq. (7) is read
 * with a plus sign, omega = 2 c_s^2 / (2 nu + c_s^2), which is Eq. (4) solved for
 * omega (the printed minus sign contradicts Eq. (4)).                          */
double or_omega_eff(double rho_r, double rho_b, double tau_r, double tau_b) {
    double nu_r = CS2 * (tau_r - 0.5), nu_b = CS2 * (tau_b - 0.5);
    double rho = rho_r + rho_b;
    double inv_nu = (rho_r / rho) / nu_r + (rho_b / rho) / nu_b;
    double nu = 1.0 / inv_nu;
    return 2.0 * CS2 / (2.0 * nu + CS2);
}

/* Eq. (1) with Eqs. (5)-(6): BGK relaxation of the total population
 * f_i = f_i^r + f_i^b towards f^eq(rho, u), u = j / rho, plus the EDM source of
 * the total force. Summing Eqs. (5) and (6) gives exactly this, because f^eq is
 * linear in the density and both species relax at omega_eff with the common u;
 * the per-species split is fixed afterwards by recolouring. The force is split
 * between species in proportion to density, F^k = (rho_k/rho) F, so that the
 * velocity shift F^k/rho^k = F/rho is common to both species.                 */
void or_bgk_edm(const double f[Q], double omega, const double F[3], double out[Q]) {
    lattice_init();
    double rho = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        j[0] += f[i] * CX[i];
        j[1] += f[i] * CY[i];
        j[2] += f[i] * CZ[i];
    }
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    double feq[Q], S[Q];
    or_feq(rho, u, feq);
    or_edm_source(rho, u, F, S);
    for (int i = 0; i < Q; ++i) out[i] = (1.0 - omega) * f[i] + omega * feq[i] + S[i];
}

/* Colour-gradient perturbation (the paper is silent; reading: the generalised
 * perturbation operator of the cited colour-gradient model, in its D3Q19 form)
 *   Delta_i = (A/2) |G| [ w_i (c_i.G)^2/|G|^2 - B_i ],  A = 9 omega sigma / 2,
 * with B_0 = -2/9, B_face = 1/54, B_edge = 1/27, applied once to the total
 * population. It conserves mass and momentum and adds the capillary stress
 * (A/9)|G| (n n - I) to the second moment, so the surface tension is
 * sigma = 2A/(9 omega) for a colour field phi running from -1 to +1.
 * Skipped where |G| < 1e-6 (reading: zero-gradient tie-break; the threshold sits
 * above the rounding level of a single-precision evaluation of the stencil on an
 * O(1) colour field, so that FP32 implementations take the same branch).       */
void or_perturb(const double f[Q], double omega, double sigma, const double G[3],
                double out[Q]) {
    lattice_init();
    double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    double gm = sqrt(g2);
    if (gm < 1e-6) {
        for (int i = 0; i < Q; ++i) out[i] = f[i];
        return;
    }
    double A = 4.5 * omega * sigma;
    for (int i = 0; i < Q; ++i) {
        double cg = CX[i] * G[0] + CY[i] * G[1] + CZ[i] * G[2];
        out[i] = f[i] + 0.5 * A * gm * (W[i] * cg * cg / g2 - BPERT[i]);
    }
}

/* Recolouring (the paper is silent; reading: Latva-Kokko & Rothman segregation)
 *   f_i^r = (rho_r/rho) f_i + beta (rho_r rho_b / rho) w_i cos(theta_i)
 *   f_i^b = (rho_b/rho) f_i - beta (rho_r rho_b / rho) w_i cos(theta_i)
 * cos(theta_i) = c_i.G / (|c_i| |G|), cos(theta_0) = 0; the beta term is
 * skipped where |G| < 1e-6 (same tie-break as the perturbation).              */
void or_recolour(const double f[Q], double rho_r, double rho_b, double beta,
                 const double G[3], double out_r[Q], double out_b[Q]) {
    lattice_init();
    double rho = rho_r + rho_b;
    double gm = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
    for (int i = 0; i < Q; ++i) {
        double seg = 0.0;
        if (gm >= 1e-6 && i != 0) {
            double cn = sqrt((double)(CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i]));
            double cosv = (CX[i] * G[0] + CY[i] * G[1] + CZ[i] * G[2]) / (cn * gm);
            seg = beta * (rho_r * rho_b / rho) * W[i] * cosv;
        }
        out_r[i] = (rho_r / rho) * f[i] + seg;
        out_b[i] = (rho_b / rho) * f[i] - seg;
    }
}

/* ------------------------------------------------------------------------- */
/* Shan-Chen binary mixture (Sec. "Multi-component flows", Eqs. (5)-(9), (12)):
 * each species relaxes by BGK at the mixture rate omega_eff towards f^eq(rho_k, u)
 * with the common velocity u = j / rho, plus its own EDM source
 * S^k = f^eq(rho_k, u + F^k/rho_k) - f^eq(rho_k, u), where F^k is the cohesive
 * force of Eq. (12) plus the species' share (rho_k/rho) F_body of the body force.
 * Reading of Eq. (12): the text makes G_C > 0 repulsive, which needs the sign of
 * the usual Shan-Chen form, F^r(x) = -G_C rho_r(x) sum_i w_i rho_b(x + c_i) c_i
 * (and F^b with the species swapped); the printed formula has no minus sign. A
 * neighbour beyond a wall takes the node's own density (neutral wall, as for the
 * colour gradient). The velocity shift F^k/rho_k is formed without dividing by
 * rho_k, so a vanishing species stays exactly zero.                             */
static void sc_shift_node(const or_params* p, const double* rho_r, const double* rho_b, long x,
                          long y, long z, double sr[3], double sb[3]) {
    double ar[3] = {0, 0, 0}, ab[3] = {0, 0, 0};   /* sum_i w_i rho_k(x + c_i) c_i */
    long id = nidx(p, x, y, z);
    for (int i = 0; i < Q; ++i) {
        if (i == 0) continue;
        long xs = x + CX[i], ys = y + CY[i], zs = z + CZ[i];
        long nb = id;
        if (!((p->wall_y && (ys < 0 || ys >= p->ny)) || (p->wall_z && (zs < 0 || zs >= p->nz))))
            nb = nidx(p, wrap(xs, p->nx), wrap(ys, p->ny), wrap(zs, p->nz));
        ar[0] += W[i] * rho_r[nb] * CX[i];
        ar[1] += W[i] * rho_r[nb] * CY[i];
        ar[2] += W[i] * rho_r[nb] * CZ[i];
        ab[0] += W[i] * rho_b[nb] * CX[i];
        ab[1] += W[i] * rho_b[nb] * CY[i];
        ab[2] += W[i] * rho_b[nb] * CZ[i];
    }
    for (int a = 0; a < 3; ++a) {
        sr[a] = -p->G_sc * ab[a];   /* F^r / rho_r */
        sb[a] = -p->G_sc * ar[a];   /* F^b / rho_b */
    }
}

/* Collision of one node in the Shan-Chen model: species densities rho_r, rho_b,
 * their post-stream populations, the cohesive velocity shifts sr, sb (F^k/rho_k)
 * and the body force Fb. Returns the total force in F.                         */
static void sc_collide_node(const or_params* p, const double gr[Q], const double gb[Q],
                            double rr, double rb, const double sr[3], const double sb[3],
                            const double Fb[3], double out_r[Q], double out_b[Q], double F[3]) {
    double rho = rr + rb, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        j[0] += (gr[i] + gb[i]) * CX[i];
        j[1] += (gr[i] + gb[i]) * CY[i];
        j[2] += (gr[i] + gb[i]) * CZ[i];
    }
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    double omega = or_omega_eff(rr, rb, p->tau_r, p->tau_b);
    double ur[3], ub[3];
    for (int a = 0; a < 3; ++a) {
        ur[a] = u[a] + sr[a] + Fb[a] / rho;
        ub[a] = u[a] + sb[a] + Fb[a] / rho;
        F[a] = rr * sr[a] + rb * sb[a] + Fb[a];
    }
    double er0[Q], er1[Q], eb0[Q], eb1[Q];
    or_feq(rr, u, er0);
    or_feq(rr, ur, er1);
    or_feq(rb, u, eb0);
    or_feq(rb, ub, eb1);
    for (int i = 0; i < Q; ++i) {
        out_r[i] = (1.0 - omega) * gr[i] + omega * er0[i] + (er1[i] - er0[i]);
        out_b[i] = (1.0 - omega) * gb[i] + omega * eb0[i] + (eb1[i] - eb0[i]);
    }
}

/* Near-contact strength A_h[h] (Eq. (11)): equal to A for h <= h_min and decaying
 * as h^-3 beyond. Reading: the h^-3 tail is shifted and rescaled so that it is
 * continuous at h_min and reaches zero at h_cut:
 *   A_h = A [ (h_min/h)^3 - (h_min/h_cut)^3 ] / [ 1 - (h_min/h_cut)^3 ].        */
double or_A_h(double h, double A, double h_min, double h_cut) {
    if (h <= h_min) return A;
    if (h >= h_cut) return 0.0;
    double a = h_min / h, b = h_min / h_cut;
    return A * (a * a * a - b * b * b) / (1.0 - b * b * b);
}

/* Trilinear interpolation of a node field at the point (x + ox, y + oy, z + oz),
 * (x, y, z) a node and o an offset; returns 0 and leaves *v unset if the point lies
 * outside the fluid along a walled axis. The cell and the weights are taken from
 * the offset alone (floor and fraction of o), so a single-precision evaluation
 * locates the point to the precision of o rather than of x + o.                */
static int interp(const or_params* p, const double* fld, long x, long y, long z, double ox,
                  double oy, double oz, double* v) {
    long base[3] = {x, y, z};
    double off[3] = {ox, oy, oz};
    int n[3] = {p->nx, p->ny, p->nz};
    int walled[3] = {0, p->wall_y, p->wall_z};
    long i0[3], i1[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(off[a]);
        long b = base[a] + (long)fl;
        double f = off[a] - fl;
        if (walled[a]) {
            if (b < 0 || b > n[a] - 1 || (b == n[a] - 1 && f > 0.0)) return 0;
            if (n[a] == 1) {
                i0[a] = i1[a] = 0;
                fr[a] = 0.0;
                continue;
            }
            if (b == n[a] - 1) { /* exactly on the last node */
                b = n[a] - 2;
                f = 1.0;
            }
            i0[a] = b;
            i1[a] = b + 1;
            fr[a] = f;
        } else {
            i0[a] = wrap(b, n[a]);
            i1[a] = wrap(b + 1, n[a]);
            fr[a] = f;
        }
    }
    double s = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double wt = (cx ? fr[0] : 1 - fr[0]) * (cy ? fr[1] : 1 - fr[1]) *
                            (cz ? fr[2] : 1 - fr[2]);
                long id = nidx(p, cx ? i1[0] : i0[0], cy ? i1[1] : i0[1],
                               cz ? i1[2] : i0[2]);
                s += wt * fld[id];
            }
    *v = s;
    return 1;
}

/* Colour gradient of a node field at one node: G = 3 sum_i w_i c_i phi(x + c_i),
 * a neighbour beyond a wall taking phi(x) (see or_gradient).                   */
static void gradient_node(const or_params* p, const double* phi, long x, long y, long z,
                          double G[3]) {
    long id = nidx(p, x, y, z);
    double g[3] = {0, 0, 0};
    for (int i = 1; i < Q; ++i) {
        long xs = x + CX[i], ys = y + CY[i], zs = z + CZ[i];
        double v;
        if ((p->wall_y && (ys < 0 || ys >= p->ny)) || (p->wall_z && (zs < 0 || zs >= p->nz)))
            v = phi[id];
        else
            v = phi[nidx(p, wrap(xs, p->nx), wrap(ys, p->ny), wrap(zs, p->nz))];
        g[0] += W[i] * CX[i] * v;
        g[1] += W[i] * CY[i] * v;
        g[2] += W[i] * CZ[i] * v;
    }
    G[0] = 3.0 * g[0];
    G[1] = 3.0 * g[1];
    G[2] = 3.0 * g[2];
}

/* Near-contact repulsive force, Eq. (11): F_rep = -A_h[h] n delta_I.
 * The paper does not say how h, n and delta_I are evaluated. Reading:
 *  - delta_I = |G| and n = -G/|G| (outward normal of the red, phi > 0, phase), so
 *    F_rep = A_h[h] G with G the colour gradient of the current step: the force
 *    pushes each interface back into its own droplet, repulsive for both members of
 *    a close pair;
 *  - the strength A_h[h] is a property of the film around the node, measured on the
 *    colour field phi_ray of the previous step (lag 1): with G' its gradient at the
 *    node and n' = -G'/|G'|, phi_ray is sampled by trilinear interpolation at
 *    x + t n' for t = -1, -1/2, 0, ..., h_cut + 2; samples with |phi| <= 1e-5
 *    carry no sign; t_d is the first downward zero crossing (red to blue) between
 *    consecutive signed samples, t_u the first upward crossing after it, both
 *    located by linear interpolation between those samples; h = t_u - t_d;
 *  - A_h = 0 if |G'| < 1e-3, if there is no such pair of crossings, or if the ray
 *    leaves the fluid through a wall before both are found;
 *  - pinning sites (if a mask is given) act as another interface: a node with
 *    |G'| >= 1e-3 whose nearest pin (within the cube of half-width ceil(h_cut))
 *    lies at distance d gets A_h[d] added.
 * This routine returns the strength A_h at node (x, y, z).                       */
/* The same strength with the two thresholds of the reading as arguments: the
 * sign band (1e-5 in the reading) and the least lagged gradient (1e-3). Used by
 * the tests to decide whether a difference between an FP32 evaluation and this
 * one is a branch taken differently at a threshold (a sample or a gradient within
 * rounding of it), by evaluating the reading with each threshold moved by the
 * FP32 rounding bound.                                                          */
/* The same strength with the lagged gradient G' at the node given (Gin) instead of
 * evaluated from phi_ray: the tests move it by the FP32 rounding bound of its
 * stencil sum, to tell a ray direction rounded differently in FP32 (which moves the
 * samples, hence the crossings) from a wrong value.                             */
double or_nc_strength_node_g(const or_params* p, const double* phi_ray,
                             const unsigned char* pin, long x, long y, long z,
                             double band, double g_min, const double* Gin);

double or_nc_strength_node_thr(const or_params* p, const double* phi_ray,
                               const unsigned char* pin, long x, long y, long z,
                               double band, double g_min) {
    lattice_init();
    double G[3];
    gradient_node(p, phi_ray, x, y, z, G);
    return or_nc_strength_node_g(p, phi_ray, pin, x, y, z, band, g_min, G);
}

double or_nc_strength_node_g(const or_params* p, const double* phi_ray,
                             const unsigned char* pin, long x, long y, long z,
                             double band, double g_min, const double* Gin) {
    lattice_init();
    if (p->A_nc == 0.0) return 0.0;
    const double G[3] = {Gin[0], Gin[1], Gin[2]};
    double gm = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
    if (!(gm >= g_min) || !isfinite(gm)) return 0.0;   /* non-finite fields: no force */
    double n[3] = {-G[0] / gm, -G[1] / gm, -G[2] / gm};
    int nsamp = (int)floor(2.0 * (p->h_cut + 3.0)) + 1; /* t = -1 ... h_cut + 2 */
    /* A sample carries a sign only if |phi| > band (samples at rounding level of
     * zero are skipped); a crossing lies between the last signed sample and the
     * next one of opposite sign, located by linear interpolation between them.  */
    double t_a = 0, v_a = 0, t_d = 0, t_u = 0;
    int have_a = 0, have_d = 0, have_u = 0;
    for (int s = 0; s < nsamp && !have_u; ++s) {
        double t = -1.0 + 0.5 * s;
        double v;
        if (!interp(p, phi_ray, x, y, z, t * n[0], t * n[1], t * n[2], &v)) break;
        if (fabs(v) <= band) continue;
        if (have_a) {
            if (!have_d && v_a > 0.0 && v < 0.0) {
                t_d = t_a + (t - t_a) * v_a / (v_a - v);
                have_d = 1;
            } else if (have_d && v_a < 0.0 && v > 0.0) {
                t_u = t_a + (t - t_a) * v_a / (v_a - v);
                have_u = 1;
            }
        }
        t_a = t;
        v_a = v;
        have_a = 1;
    }
    double Ah = 0.0;
    if (have_d && have_u) Ah = or_A_h(t_u - t_d, p->A_nc, p->h_min, p->h_cut);
    if (pin) {
        int r = (int)ceil(p->h_cut);
        double best = -1.0;
        for (int dz = -r; dz <= r; ++dz)
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    long xs = x + dx, ys = y + dy, zs = z + dz;
                    if (p->wall_y && (ys < 0 || ys >= p->ny)) continue;
                    if (p->wall_z && (zs < 0 || zs >= p->nz)) continue;
                    xs = wrap(xs, p->nx);
                    ys = wrap(ys, p->ny);
                    zs = wrap(zs, p->nz);
                    if (!pin[nidx(p, xs, ys, zs)]) continue;
                    double d = sqrt((double)(dx * dx + dy * dy + dz * dz));
                    if (best < 0 || d < best) best = d;
                }
        if (best >= 0) Ah += or_A_h(best, p->A_nc, p->h_min, p->h_cut);
    }
    return Ah;
}

double or_nc_strength_node(const or_params* p, const double* phi_ray,
                           const unsigned char* pin, long x, long y, long z) {
    return or_nc_strength_node_thr(p, phi_ray, pin, x, y, z, 1e-5, 1e-3);
}

/* Isotropic colour gradient G(x) = 3 sum_i w_i c_i phi(x + c_i), the stencil form
 * the paper uses for the inter-component force, Eq. (10). Reading at walls: a
 * neighbour outside the fluid takes phi(x) (neutral wetting).                  */
void or_gradient(const or_params* p, const double* phi, double* Gx, double* Gy,
                 double* Gz) {
    lattice_init();
#pragma omp parallel for schedule(static)
    for (long z = 0; z < p->nz; ++z)
        for (long y = 0; y < p->ny; ++y)
            for (long x = 0; x < p->nx; ++x) {
                long id = nidx(p, x, y, z);
                double g[3] = {0, 0, 0};
                for (int i = 1; i < Q; ++i) {
                    long xs = x + CX[i], ys = y + CY[i], zs = z + CZ[i];
                    double v;
                    if ((p->wall_y && (ys < 0 || ys >= p->ny)) ||
                        (p->wall_z && (zs < 0 || zs >= p->nz)))
                        v = phi[id];
                    else
                        v = phi[nidx(p, wrap(xs, p->nx), wrap(ys, p->ny), wrap(zs, p->nz))];
                    g[0] += W[i] * CX[i] * v;
                    g[1] += W[i] * CY[i] * v;
                    g[2] += W[i] * CZ[i] * v;
                }
                Gx[id] = 3.0 * g[0];
                Gy[id] = 3.0 * g[1];
                Gz[id] = 3.0 * g[2];
            }
}

/* ------------------------------------------------------------------------- */
/* State management.                                                          */
or_state* or_create(const or_params* p) {
    lattice_init();
    or_state* s = (or_state*)calloc(1, sizeof(or_state));
    if (!s) return NULL;
    s->p = *p;
    s->N = (long)p->nx * p->ny * p->nz;
    long N = s->N;
    double** bufs[] = {&s->fr, &s->fb, &s->gr, &s->gb};
    for (int b = 0; b < 4; ++b) {
        *bufs[b] = (double*)calloc((size_t)Q * N, sizeof(double));
        if (!*bufs[b]) return NULL;
    }
    double** f1[] = {&s->rho_r, &s->rho_b, &s->jx, &s->jy, &s->jz, &s->phi, &s->phi_lag,
                     &s->Gx, &s->Gy, &s->Gz, &s->Fx, &s->Fy, &s->Fz};
    for (int b = 0; b < 13; ++b) {
        *f1[b] = (double*)calloc((size_t)N, sizeof(double));
        if (!*f1[b]) return NULL;
    }
    return s;
}

void or_destroy(or_state* s) {
    if (!s) return;
    double* all[] = {s->fr, s->fb, s->gr, s->gb, s->rho_r, s->rho_b, s->jx, s->jy, s->jz,
                     s->phi, s->phi_lag, s->Gx, s->Gy, s->Gz, s->Fx, s->Fy, s->Fz};
    for (int b = 0; b < 17; ++b) free(all[b]);
    free(s->pin);
    free(s);
}

/* Initial state f_i^k = f_i^eq(rho_k, u), Eq. (2); u may be NULL (= 0). The
 * moment arrays and both colour-field buffers are set from the given fields.  */
void or_set_fields(or_state* s, const double* rho_r, const double* rho_b, const double* u) {
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        double uu[3] = {0, 0, 0};
        if (u) {
            uu[0] = u[n];
            uu[1] = u[N + n];
            uu[2] = u[2 * N + n];
        }
        double er[Q], eb[Q];
        or_feq(rho_r[n], uu, er);
        or_feq(rho_b[n], uu, eb);
        for (int i = 0; i < Q; ++i) {
            s->fr[(long)i * N + n] = er[i];
            s->fb[(long)i * N + n] = eb[i];
        }
        double rho = rho_r[n] + rho_b[n];
        s->rho_r[n] = rho_r[n];
        s->rho_b[n] = rho_b[n];
        s->jx[n] = rho * uu[0];
        s->jy[n] = rho * uu[1];
        s->jz[n] = rho * uu[2];
        s->Fx[n] = s->Fy[n] = s->Fz[n] = 0.0;
        s->phi[n] = (rho_r[n] - rho_b[n]) / rho;
        s->phi_lag[n] = s->phi[n];
    }
    s->steps = 0;
}

void or_set_pins(or_state* s, const unsigned char* mask) {
    free(s->pin);
    s->pin = NULL;
    if (!mask) return;
    s->pin = (unsigned char*)malloc((size_t)s->N);
    memcpy(s->pin, mask, (size_t)s->N);
}

/* Raw populations in and out, layout [i][N] per species. */
void or_get_pops(const or_state* s, double* fr, double* fb) {
    memcpy(fr, s->fr, sizeof(double) * Q * s->N);
    memcpy(fb, s->fb, sizeof(double) * Q * s->N);
}
void or_set_pops(or_state* s, const double* fr, const double* fb, const double* phi_lag) {
    memcpy(s->fr, fr, sizeof(double) * Q * s->N);
    memcpy(s->fb, fb, sizeof(double) * Q * s->N);
    if (phi_lag) memcpy(s->phi_lag, phi_lag, sizeof(double) * s->N);
}
void or_get_phi_lag(const or_state* s, double* phi_lag) {
    memcpy(phi_lag, s->phi_lag, sizeof(double) * s->N);
}

/* Pull streaming of one node (Eq. (1) read from the receiving side; streaming is
 * a pure memory shift). A source x - c_i outside the fluid along a walled axis
 * means the population left x towards the wall and came back: halfway
 * bounce-back, f_i(x, t+1) = f*_{opp(i)}(x, t). x is always periodic.          */
static void pull_node(const or_params* p, long N, const double* fr, const double* fb,
                      long x, long y, long z, double gr[Q], double gb[Q]) {
    for (int i = 0; i < Q; ++i) {
        long xs = x - CX[i], ys = y - CY[i], zs = z - CZ[i];
        if ((p->wall_y && (ys < 0 || ys >= p->ny)) || (p->wall_z && (zs < 0 || zs >= p->nz))) {
            long id = nidx(p, x, y, z);
            gr[i] = fr[(long)OPP[i] * N + id];
            gb[i] = fb[(long)OPP[i] * N + id];
        } else {
            long id = nidx(p, wrap(xs, p->nx), wrap(ys, p->ny), wrap(zs, p->nz));
            gr[i] = fr[(long)i * N + id];
            gb[i] = fb[(long)i * N + id];
        }
    }
}

/* Sliding walls (Sec. "High-performance LB code for bijel materials": a bijel
 * confined between walls moving in opposite directions, +-U along the periodic
 * axis). Reading: halfway bounce-back from a wall moving with velocity u_w adds
 * 2 w_i rho (c_i . u_w)/c_s^2 = 6 w_i rho (c_i . u_w) to the reflected population
 * (the moving-wall bounce-back of Ladd), per species with that species' density
 * at the node. The terms of the links arriving from one wall sum to zero
 * (sum of w_i c_ix over them vanishes), so the densities are those of the plain
 * bounce-back, which is what they are computed from. Applied to the post-stream
 * populations of a node at y = 0 or ny - 1 (walled y axis).                      */
static void moving_wall(const or_params* p, long y, double gr[Q], double gb[Q]) {
    if (!p->wall_y || p->wall_u == 0.0) return;
    double rr = 0.0, rb = 0.0;
    for (int i = 0; i < Q; ++i) {
        rr += gr[i];
        rb += gb[i];
    }
    for (int i = 0; i < Q; ++i) {
        long ys = y - CY[i];
        double uw;
        if (ys >= p->ny) uw = p->wall_u;        /* from the wall at y = ny - 1/2 */
        else if (ys < 0) uw = -p->wall_u;       /* from the wall at y = -1/2     */
        else continue;
        double cu = CX[i] * uw;
        gr[i] += 2.0 * W[i] * rr * cu / CS2;
        gb[i] += 2.0 * W[i] * rb * cu / CS2;
    }
}

/* Streaming alone (no collision), for the exact-permutation check. */
void or_stream_only(or_state* s, int nsteps) {
    const or_params* p = &s->p;
    long N = s->N;
    for (int t = 0; t < nsteps; ++t) {
#pragma omp parallel for schedule(static)
        for (long z = 0; z < p->nz; ++z)
            for (long y = 0; y < p->ny; ++y)
                for (long x = 0; x < p->nx; ++x) {
                    double a[Q], b[Q];
                    long id = nidx(p, x, y, z);
                    pull_node(p, N, s->fr, s->fb, x, y, z, a, b);
                    for (int i = 0; i < Q; ++i) {
                        s->gr[(long)i * N + id] = a[i];
                        s->gb[(long)i * N + id] = b[i];
                    }
                }
        double* t1 = s->fr; s->fr = s->gr; s->gr = t1;
        double* t2 = s->fb; s->fb = s->gb; s->gb = t2;
    }
}

/* Body force density at row y: uniform g plus the Kolmogorov profile. Reading:
 * g is a force density (F = g, not rho g).                                      */
static void body_force(const or_params* p, long y, double F[3]) {
    F[0] = p->g[0] + p->kolmogorov_amp * sin(2.0 * M_PI * (double)y / (double)p->ny);
    F[1] = p->g[1];
    F[2] = p->g[2];
}

/* Collision, perturbation and recolouring of one node from its post-stream
 * populations, moments, colour gradient and force.                             */
static void collide_node(const or_params* p, const double gr[Q], const double gb[Q],
                         double rho_r, double rho_b, const double G[3], const double F[3],
                         double out_r[Q], double out_b[Q]) {
    double f[Q], f1[Q], f2[Q];
    for (int i = 0; i < Q; ++i) f[i] = gr[i] + gb[i];
    double omega = or_omega_eff(rho_r, rho_b, p->tau_r, p->tau_b);
    or_bgk_edm(f, omega, F, f1);
    or_perturb(f1, omega, p->sigma, G, f2);
    or_recolour(f2, rho_r, rho_b, p->beta, G, out_r, out_b);
}

/* One full time step, phases 1..7 in order (see the file header). */
void or_step(or_state* s, int nsteps) {
    const or_params* p = &s->p;
    long N = s->N;
    for (int t = 0; t < nsteps; ++t) {
        /* 1. streaming */
#pragma omp parallel for schedule(static)
        for (long z = 0; z < p->nz; ++z)
            for (long y = 0; y < p->ny; ++y)
                for (long x = 0; x < p->nx; ++x) {
                    double a[Q], b[Q];
                    long id = nidx(p, x, y, z);
                    pull_node(p, N, s->fr, s->fb, x, y, z, a, b);
                    moving_wall(p, y, a, b);
                    for (int i = 0; i < Q; ++i) {
                        s->gr[(long)i * N + id] = a[i];
                        s->gb[(long)i * N + id] = b[i];
                    }
                }
        /* 2. moments, Eq. (3), and the colour field phi = (rho_r - rho_b)/rho */
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            double rr = 0, rb = 0, j[3] = {0, 0, 0};
            for (int i = 0; i < Q; ++i) {
                double a = s->gr[(long)i * N + n], b = s->gb[(long)i * N + n];
                rr += a;
                rb += b;
                j[0] += (a + b) * CX[i];
                j[1] += (a + b) * CY[i];
                j[2] += (a + b) * CZ[i];
            }
            s->rho_r[n] = rr;
            s->rho_b[n] = rb;
            s->jx[n] = j[0];
            s->jy[n] = j[1];
            s->jz[n] = j[2];
            s->phi[n] = (rr - rb) / (rr + rb);
        }
        if (p->model == 1) {
            /* Shan-Chen: 3'. cohesive forces from the densities of this step, and
             * 5'. per-species BGK + EDM (no perturbation, no recolouring) */
#pragma omp parallel for schedule(static)
            for (long z = 0; z < p->nz; ++z)
                for (long y = 0; y < p->ny; ++y)
                    for (long x = 0; x < p->nx; ++x) {
                        long id = nidx(p, x, y, z);
                        double a[Q], b[Q], oa[Q], ob[Q], sr[3], sb[3], Fb[3], F[3];
                        for (int i = 0; i < Q; ++i) {
                            a[i] = s->gr[(long)i * N + id];
                            b[i] = s->gb[(long)i * N + id];
                        }
                        sc_shift_node(p, s->rho_r, s->rho_b, x, y, z, sr, sb);
                        body_force(p, y, Fb);
                        sc_collide_node(p, a, b, s->rho_r[id], s->rho_b[id], sr, sb, Fb, oa, ob, F);
                        s->Fx[id] = F[0];
                        s->Fy[id] = F[1];
                        s->Fz[id] = F[2];
                        for (int i = 0; i < Q; ++i) {
                            s->fr[(long)i * N + id] = oa[i];
                            s->fb[(long)i * N + id] = ob[i];
                        }
                    }
            memcpy(s->phi_lag, s->phi, sizeof(double) * N);
            s->steps++;
            continue;
        }
        /* 3. colour gradient */
        or_gradient(p, s->phi, s->Gx, s->Gy, s->Gz);
        /* 4. forces */
        const double* phi_ray = p->nc_lag ? s->phi_lag : s->phi;
#pragma omp parallel for schedule(static)
        for (long z = 0; z < p->nz; ++z)
            for (long y = 0; y < p->ny; ++y)
                for (long x = 0; x < p->nx; ++x) {
                    long id = nidx(p, x, y, z);
                    double Fb[3], Fn[3];
                    double G[3] = {s->Gx[id], s->Gy[id], s->Gz[id]};
                    body_force(p, y, Fb);
                    double ah = or_nc_strength_node(p, phi_ray, s->pin, x, y, z);
                    for (int a = 0; a < 3; ++a) Fn[a] = ah * G[a];
                    s->Fx[id] = Fb[0] + Fn[0];
                    s->Fy[id] = Fb[1] + Fn[1];
                    s->Fz[id] = Fb[2] + Fn[2];
                }
        /* 5.-7. collision + EDM, perturbation, recolouring; result is the new state */
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            double a[Q], b[Q], oa[Q], ob[Q];
            for (int i = 0; i < Q; ++i) {
                a[i] = s->gr[(long)i * N + n];
                b[i] = s->gb[(long)i * N + n];
            }
            double G[3] = {s->Gx[n], s->Gy[n], s->Gz[n]};
            double F[3] = {s->Fx[n], s->Fy[n], s->Fz[n]};
            collide_node(p, a, b, s->rho_r[n], s->rho_b[n], G, F, oa, ob);
            for (int i = 0; i < Q; ++i) {
                s->fr[(long)i * N + n] = oa[i];
                s->fb[(long)i * N + n] = ob[i];
            }
        }
        /* this step's colour field is the next step's lagged field */
        memcpy(s->phi_lag, s->phi, sizeof(double) * N);
        s->steps++;
    }
}

/* Fields of the last step: rho_r, rho_b, phi and the physical velocity
 * u = (j + F/2)/rho of the EDM scheme ([3][N]). Before any step: the fields set. */
void or_get_fields(const or_state* s, double* rho_r, double* rho_b, double* u, double* phi) {
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        double rho = s->rho_r[n] + s->rho_b[n];
        if (rho_r) rho_r[n] = s->rho_r[n];
        if (rho_b) rho_b[n] = s->rho_b[n];
        if (u) {
            u[n] = (s->jx[n] + 0.5 * s->Fx[n]) / rho;
            u[N + n] = (s->jy[n] + 0.5 * s->Fy[n]) / rho;
            u[2 * N + n] = (s->jz[n] + 0.5 * s->Fz[n]) / rho;
        }
        if (phi) phi[n] = s->phi[n];
    }
}

/* Forces of the last step ([3][N]). */
void or_get_forces(const or_state* s, double* F) {
    long N = s->N;
    memcpy(F, s->Fx, sizeof(double) * N);
    memcpy(F + N, s->Fy, sizeof(double) * N);
    memcpy(F + 2 * N, s->Fz, sizeof(double) * N);
}

/* Neumaier compensated summation: the conservation checks compare totals of
 * ~10^6 terms to 1e-12 relative, below the error of a naive running sum.      */
typedef struct { double s, c; } ksum;
static inline void kadd(ksum* k, double v) {
    double t = k->s + v;
    if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
    else k->c += (v - t) + k->s;
    k->s = t;
}

/* Conserved totals of the state, in node order:
 * out = {sum f^r, sum f^b, P_x, P_y, P_z} with P = sum_i c_i (f^r_i + f^b_i).   */
void or_totals(const or_state* s, double out[5]) {
    long N = s->N;
    ksum k[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (long n = 0; n < N; ++n)
        for (int i = 0; i < Q; ++i) {
            double a = s->fr[(long)i * N + n], b = s->fb[(long)i * N + n];
            kadd(&k[0], a);
            kadd(&k[1], b);
            kadd(&k[2], (a + b) * CX[i]);
            kadd(&k[3], (a + b) * CY[i]);
            kadd(&k[4], (a + b) * CZ[i]);
        }
    for (int a = 0; a < 5; ++a) out[a] = k[a].s + k[a].c;
}

/* One step evaluated at a list of nodes only, from a given input state
 * (populations fr, fb [i][N] and lagged colour field phi_lag). Same definition
 * as or_step, restricted: the colour field at the 18 neighbours of each listed
 * node is rebuilt from their own pulled populations. Writes the new populations
 * of the listed nodes to out_r, out_b ([nlist][Q]) and their force to F ([nlist][3]).
 * The near-contact ray needs the current colour field only when nc_lag == 0,
 * which this routine does not support (returns -1).                           */
static int step_nodes_impl(const or_params* p, const double* fr, const double* fb,
                           const double* phi_lag, const unsigned char* pin, long nlist,
                           const long* list, const double* ah_given, double* out_r,
                           double* out_b, double* Fout) {
    lattice_init();
    if (!p->nc_lag && p->A_nc != 0.0) return -1;
    long N = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(dynamic, 64)
    for (long k = 0; k < nlist; ++k) {
        long id = list[k];
        long x = id % p->nx, y = (id / p->nx) % p->ny, z = id / ((long)p->nx * p->ny);
        double gr[Q], gb[Q];
        pull_node(p, N, fr, fb, x, y, z, gr, gb);
        moving_wall(p, y, gr, gb);
        double rr = 0, rb = 0;
        for (int i = 0; i < Q; ++i) {
            rr += gr[i];
            rb += gb[i];
        }
        double phi0 = (rr - rb) / (rr + rb);
        double g[3] = {0, 0, 0};
        double ar[3] = {0, 0, 0}, ab[3] = {0, 0, 0};   /* Shan-Chen density sums */
        for (int i = 1; i < Q; ++i) {
            long xs = x + CX[i], ys = y + CY[i], zs = z + CZ[i];
            double v, nr = rr, nb = rb;
            if ((p->wall_y && (ys < 0 || ys >= p->ny)) || (p->wall_z && (zs < 0 || zs >= p->nz))) {
                v = phi0;
            } else {
                double hr[Q], hb[Q], sr = 0, sb = 0;
                pull_node(p, N, fr, fb, wrap(xs, p->nx), wrap(ys, p->ny), wrap(zs, p->nz), hr,
                          hb);
                for (int m = 0; m < Q; ++m) {
                    sr += hr[m];
                    sb += hb[m];
                }
                v = (sr - sb) / (sr + sb);
                nr = sr;
                nb = sb;
            }
            g[0] += W[i] * CX[i] * v;
            g[1] += W[i] * CY[i] * v;
            g[2] += W[i] * CZ[i] * v;
            ar[0] += W[i] * nr * CX[i];
            ar[1] += W[i] * nr * CY[i];
            ar[2] += W[i] * nr * CZ[i];
            ab[0] += W[i] * nb * CX[i];
            ab[1] += W[i] * nb * CY[i];
            ab[2] += W[i] * nb * CZ[i];
        }
        if (p->model == 1) {
            double sr3[3], sb3[3], Fb[3], F[3];
            for (int a = 0; a < 3; ++a) {
                sr3[a] = -p->G_sc * ab[a];
                sb3[a] = -p->G_sc * ar[a];
            }
            body_force(p, y, Fb);
            sc_collide_node(p, gr, gb, rr, rb, sr3, sb3, Fb, out_r + k * Q, out_b + k * Q, F);
            if (Fout)
                for (int a = 0; a < 3; ++a) Fout[3 * k + a] = F[a];
            continue;
        }
        double G[3] = {3.0 * g[0], 3.0 * g[1], 3.0 * g[2]};
        double Fb[3], Fn[3], F[3];
        body_force(p, y, Fb);
        double ah = ah_given ? ah_given[k] : or_nc_strength_node(p, phi_lag, pin, x, y, z);
        for (int a = 0; a < 3; ++a) Fn[a] = ah * G[a];
        for (int a = 0; a < 3; ++a) F[a] = Fb[a] + Fn[a];
        collide_node(p, gr, gb, rr, rb, G, F, out_r + k * Q, out_b + k * Q);
        if (Fout)
            for (int a = 0; a < 3; ++a) Fout[3 * k + a] = F[a];
    }
    return 0;
}

int or_step_nodes(const or_params* p, const double* fr, const double* fb,
                  const double* phi_lag, const unsigned char* pin, long nlist,
                  const long* list, double* out_r, double* out_b, double* Fout) {
    return step_nodes_impl(p, fr, fb, phi_lag, pin, nlist, list, NULL, out_r, out_b, Fout);
}

/* The same step at the listed nodes with the near-contact strength A_h of each
 * listed node given (ah[k] for list[k]) instead of measured: the tests use it to
 * follow a node whose film measurement took the other branch at a threshold.   */
int or_step_nodes_given_ah(const or_params* p, const double* fr, const double* fb,
                           const double* phi_lag, const unsigned char* pin, long nlist,
                           const long* list, const double* ah, double* out_r, double* out_b,
                           double* Fout) {
    return step_nodes_impl(p, fr, fb, phi_lag, pin, nlist, list, ah, out_r, out_b, Fout);
}

/* Laplace-law measurement (static droplet): with phi and rho taken from the state
 * (sums of the post-collision populations), V = sum (1 + phi)/2,
 * R_eff = (3V/(4 pi))^(1/3), p = rho c_s^2; p_in is the mean over nodes with
 * r < R_eff - 3 and p_out the mean over r > R_eff + 5, r being the
 * minimum-image distance to the centre c along periodic axes.
 * out = {dp, R_eff, p_in, p_out, V}.                                           */
void or_laplace(const or_state* s, const double c[3], double out[5]) {
    const or_params* p = &s->p;
    long N = s->N;
    double V = 0;
    double* rho = (double*)malloc(sizeof(double) * N);
    for (long n = 0; n < N; ++n) {
        double rr = 0, rb = 0;
        for (int i = 0; i < Q; ++i) {
            rr += s->fr[(long)i * N + n];
            rb += s->fb[(long)i * N + n];
        }
        rho[n] = rr + rb;
        V += 0.5 * (1.0 + (rr - rb) / (rr + rb));
    }
    double R = cbrt(3.0 * V / (4.0 * M_PI));
    double sin_ = 0, sout = 0;
    long nin = 0, nout = 0;
    int n3[3] = {p->nx, p->ny, p->nz};
    int per[3] = {1, !p->wall_y, !p->wall_z};
    for (long z = 0; z < p->nz; ++z)
        for (long y = 0; y < p->ny; ++y)
            for (long x = 0; x < p->nx; ++x) {
                double d[3] = {x - c[0], y - c[1], z - c[2]};
                for (int a = 0; a < 3; ++a)
                    if (per[a]) {
                        if (d[a] > 0.5 * n3[a]) d[a] -= n3[a];
                        if (d[a] < -0.5 * n3[a]) d[a] += n3[a];
                    }
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                long id = nidx(p, x, y, z);
                if (r < R - 3.0) {
                    sin_ += rho[id] * CS2;
                    nin++;
                } else if (r > R + 5.0) {
                    sout += rho[id] * CS2;
                    nout++;
                }
            }
    free(rho);
    double pin_ = nin ? sin_ / nin : NAN, pout = nout ? sout / nout : NAN;
    out[0] = pin_ - pout;
    out[1] = R;
    out[2] = pin_;
    out[3] = pout;
    out[4] = V;
}
