/*
 * oracle.c -- plain, slow, FP64 CPU restatement of one time step of the hybrid
 * lattice-Boltzmann / dynamic self-consistent-field (DSCF) method of Zhang, Sevink and
 * Schmid, "Hybrid Lattice Boltzmann / Dynamic Self-Consistent Field Simulations of
 * Microphase Separation and Vesicle Formation in Block Copolymer Systems" (arXiv:1204.2088).
 *
 * TEST INFRASTRUCTURE.  This file is the checker, not the product: only the test-suite,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or helper with the CUDA library; the two agree only through the
 * equations of the paper and the readings listed with each function below.
 *
 * Every loop is written in the order of the definition it follows; the only liberty taken
 * is an OpenMP "parallel for" over independent lattice sites.  All reductions are serial
 * (fixed order) so the oracle is deterministic.
 *
 * Conventions (shared with the CUDA side only as documented conventions):
 *   - lattice spacing h = 1, energies in k_B T, time in tau = h^2/(k_B T M)   (Sec. 2, units)
 *   - fields are stored x fastest: idx = x + nx*(y + ny*z), species-major [I][V]
 *   - species order A, B, S
 *   - D3Q19 velocity order: 0:(000); 1..6: +x,-x,+y,-y,+z,-z;
 *     7..18: (+x+y) (-x-y) (+x-y) (-x+y) (+x+z) (-x-z) (+x-z) (-x+z) (+y+z) (-y-z) (+y-z) (-y+z)
 *   - LB runs in lattice units (Delta t_LB = 1, c = 1, c_s^2 = 1/3, rho0 = 1); the thermodynamic
 *     force enters as f_lat = dt^2 * f and the LB velocity u_lat = dt * u is the Courant number
 *     the convection step uses.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz;
    int32_t ns;          /* 2 = A,B melt; 3 = A,B copolymer + single-bead solvent S      */
    int32_t N, nA;       /* beads per chain N_p and A-block length n (bead s is A if s<=nA) */
    double phi_p;        /* mean copolymer volume fraction (1 in a melt)                 */
    double chi[9];       /* Flory-Huggins chi_IJ, row-major 3x3, zero diagonal           */
    double kappa;        /* Helfand kappa_H v0 / k_B T                                  */
    double a;            /* statistical segment length in units of h                    */
    double dt, M;        /* time step (tau) and mobility                                */
    double tau_s, tau_b; /* LB shear / bulk relaxation times (lattice units)            */
    double rho0;         /* LB reference mass density                                   */
    int32_t hydro;       /* 0: diffusion only (u = 0), 1: LB coupled                    */
    int32_t ncg_iters;   /* Fletcher-Reeves iterations per time step                     */
    int32_t cn_sweeps;   /* Jacobi sweeps for the Crank-Nicolson system                  */
    double phi_floor;    /* floor on phi inside the local curvature of mu              */
    double ncg_tol;      /* > 0: stop the inversion once max|phi* - phi[U]| < ncg_tol    */
    double omega;        /* > 0: thermal noise with noise parameter Omega = h^3/v0        */
    int32_t lb_noise;    /* with omega > 0: also the fluctuating LB modes (Eq. 13)       */
    int32_t warm_extrap; /* 1: start the inversion from 2 U^{n-1} - U^{n-2} (or_step)      */
    uint64_t seed;       /* key of the counter-based generator                           */
    int64_t step;        /* step index (counter word 1) of the noise of this call        */
} or_params;

static inline int64_t nsites(const or_params* p) { return (int64_t)p->nx * p->ny * p->nz; }
static inline int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }
static inline int64_t sidx(const or_params* p, int x, int y, int z) {
    return (int64_t)wrap(x, p->nx) + (int64_t)p->nx * ((int64_t)wrap(y, p->ny) + (int64_t)p->ny * wrap(z, p->nz));
}

/* ------------------------------------------------------------------------------------ */
/* Linkage operator sigma (Sec. 2, Eq. 17 and the Gaussian kernel after it).             */
/* Reading: the 27-point stencil is the tensor product of a 1-D three-point kernel        */
/* (alpha, 1-2*alpha, alpha) whose variance 2*alpha*h^2 equals the per-axis variance a^2/3 */
/* of a Gaussian bond; the weights therefore sum to one (sigma[1] = 1).                  */
/* w[0] centre, w[1] face (6), w[2] edge (12), w[3] corner (8).                           */
/* ------------------------------------------------------------------------------------ */
void or_stencil_weights(double a, double w[4]) {
    double alpha = a * a / 6.0;
    double beta = 1.0 - 2.0 * alpha;
    w[0] = beta * beta * beta;
    w[1] = alpha * beta * beta;
    w[2] = alpha * alpha * beta;
    w[3] = alpha * alpha * alpha;
}

/* sigma[f](r) = sum over the 27 offsets o of w(|o|_1) f(r + o), periodic. */
void or_sigma(const or_params* p, const double* f, double* out) {
    double w[4];
    or_stencil_weights(p->a, w);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double acc = 0.0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int cls = abs(dx) + abs(dy) + abs(dz);
                            acc += w[cls] * f[sidx(p, x + dx, y + dy, z + dz)];
                        }
                out[sidx(p, x, y, z)] = acc;
            }
}

/* ------------------------------------------------------------------------------------ */
/* Densities from the potentials (Eq. 2 via the Green-propagator form Eq. 16-17).         */
/*   G_0 = 1,       G_s  = exp(-U_{I_s}) sigma[G_{s-1}],      s = 1..N                    */
/*   G+_{N+1} = 1,  G+_s = exp(-U_{I_s}) sigma[G+_{s+1}],     s = N..1                    */
/*   rho_I(r) ~ sum_{s in I} G_s(r) sigma[G+_{s+1}](r)                                   */
/* Normalisation (Eq. 2, prefactor n_p/Phi_p) in volume fractions:                        */
/*   phi_I = phi_p / (N Q) * sum_{s in I} G_s sigma[G+_{s+1}],  Q = V^-1 sum_r G_N(r)     */
/* Solvent (Eq. 2, third line): phi_S = phi_s exp(-U_S) / <exp(-U_S)>.                    */
/* Returns Q; *QS (if non-NULL) receives <exp(-U_S)> (1 in a melt).                       */
/* Gstack (optional, (N+1)*V) receives G_0..G_N.                                          */
/* ------------------------------------------------------------------------------------ */
double or_densities(const or_params* p, const double* U, double* phi, double* QS, double* Gstack) {
    const int64_t V = nsites(p);
    const int N = p->N;
    double* G = Gstack ? Gstack : (double*)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)V);
    double* Gp = (double*)malloc(sizeof(double) * (size_t)V);     /* G+_{s+1}            */
    double* sGp = (double*)malloc(sizeof(double) * (size_t)V);    /* sigma[G+_{s+1}]     */
    double* E = (double*)malloc(sizeof(double) * 2 * (size_t)V);   /* exp(-U_A), exp(-U_B) */
    for (int64_t i = 0; i < V; ++i) {
        E[i] = exp(-U[i]);
        E[V + i] = exp(-U[V + i]);
    }
    /* forward recurrence */
    for (int64_t i = 0; i < V; ++i) G[i] = 1.0;
    for (int s = 1; s <= N; ++s) {
        const double* Es = E + (s <= p->nA ? 0 : V);
        double* Gs = G + (int64_t)s * V;
        or_sigma(p, G + (int64_t)(s - 1) * V, Gs);
        for (int64_t i = 0; i < V; ++i) Gs[i] *= Es[i];
    }
    double Qsum = 0.0;
    for (int64_t i = 0; i < V; ++i) Qsum += G[(int64_t)N * V + i];
    const double Q = Qsum / (double)V;

    /* backward recurrence and contour quadrature */
    double* qA = phi;
    double* qB = phi + V;
    for (int64_t i = 0; i < V; ++i) { qA[i] = 0.0; qB[i] = 0.0; Gp[i] = 1.0; }
    for (int s = N; s >= 1; --s) {
        const double* Es = E + (s <= p->nA ? 0 : V);
        double* qI = (s <= p->nA) ? qA : qB;
        or_sigma(p, Gp, sGp);                       /* sigma[G+_{s+1}] */
        const double* Gs = G + (int64_t)s * V;
        for (int64_t i = 0; i < V; ++i) {
            qI[i] += Gs[i] * sGp[i];
            Gp[i] = Es[i] * sGp[i];                  /* becomes G+_s */
        }
    }
    const double coef = p->phi_p / ((double)N * Q);
    for (int64_t i = 0; i < V; ++i) { qA[i] *= coef; qB[i] *= coef; }

    double qs = 1.0;
    if (p->ns == 3) {
        const double* US = U + 2 * V;
        double* phS = phi + 2 * V;
        double acc = 0.0;
        for (int64_t i = 0; i < V; ++i) acc += exp(-US[i]);
        qs = acc / (double)V;
        const double phis = 1.0 - p->phi_p;
        for (int64_t i = 0; i < V; ++i) phS[i] = phis * exp(-US[i]) / qs;
    }
    if (QS) *QS = qs;
    free(E); free(sGp); free(Gp);
    if (!Gstack) free(G);
    return Q;
}

/* ------------------------------------------------------------------------------------ */
/* Objective of the self-consistent inversion (reading of Sec. 2, last paragraph: the     */
/* potentials are found with Fletcher-Reeves nonlinear CG; the objective is not printed). */
/* L(U) = (phi_p V/N) ln Q[U] + phi_s V ln <exp(-U_S)> + sum_I sum_r U_I(r) phi*_I(r)     */
/* is convex in U and its gradient is dL/dU_I(r) = phi*_I(r) - phi_I[U](r).               */
/* ------------------------------------------------------------------------------------ */
double or_objective(const or_params* p, const double* U, const double* phi_target) {
    const int64_t V = nsites(p);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)p->ns * (size_t)V);
    double qs = 1.0;
    double Q = or_densities(p, U, tmp, &qs, NULL);
    free(tmp);
    double L = p->phi_p * (double)V / (double)p->N * log(Q);
    if (p->ns == 3) L += (1.0 - p->phi_p) * (double)V * log(qs);
    for (int64_t i = 0; i < (int64_t)p->ns * V; ++i) L += U[i] * phi_target[i];
    return L;
}

static double dotv(const double* a, const double* b, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------------------------------ */
/* Fletcher-Reeves nonlinear conjugate gradient on L(U) (Sec. 2, last paragraph).        */
/* At most ncg_iters iterations; with ncg_tol > 0 the inversion also stops before an       */
/* iteration whose starting residual max|g| is below ncg_tol (or not a number).  Secant    */
/* line search with one trial point whose step comes from the local curvature             */
/* <d, phi[U] d> (the large-wavevector limit of the Hessian of L).  Per iteration k:       */
/*   h0 = <g,d>, c = <d, phi_m d>, a1 = -h0/c                   (trial step)             */
/*   h1 = <phi* - phi[U + a1 d], d>                                                        */
/*   a  = a1 * (-h0) / (h1 - h0)                                (secant root)             */
/*   U += a d;  g' = phi* - phi[U];  beta = <g',g'>/<g,g>;  d = -g' + beta d              */
/* U is updated in place; phi_model receives phi[U] at the final U.                       */
/* info (length 2 + 4*K): gg0, max|g0|, then per iteration a1, a, gg, max|g|; the entries  */
/* of iterations not run are left untouched.  Returns the number of iterations run.       */
/* ------------------------------------------------------------------------------------ */
int or_ncg(const or_params* p, const double* phi_target, double* U, double* phi_model, double* info) {
    const int64_t V = nsites(p);
    const int64_t n = (int64_t)p->ns * V;
    double* g = (double*)malloc(sizeof(double) * (size_t)n);
    double* d = (double*)malloc(sizeof(double) * (size_t)n);
    double* Ut = (double*)malloc(sizeof(double) * (size_t)n);
    double* pt = (double*)malloc(sizeof(double) * (size_t)n);

    or_densities(p, U, phi_model, NULL, NULL);
    double gmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        g[i] = phi_target[i] - phi_model[i];
        d[i] = -g[i];
        if (fabs(g[i]) > gmax) gmax = fabs(g[i]);
    }
    double gg = dotv(g, g, n);
    if (info) { info[0] = gg; info[1] = gmax; }

    int k = 0;
    for (; k < p->ncg_iters; ++k) {
        if (p->ncg_tol > 0.0 && !(gmax >= p->ncg_tol)) break;
        double h0 = dotv(g, d, n);
        double c = 0.0;
        for (int64_t i = 0; i < n; ++i) c += d[i] * phi_model[i] * d[i];
        double a1 = (c > 0.0 && isfinite(h0 / c)) ? -h0 / c : 0.0;
        for (int64_t i = 0; i < n; ++i) Ut[i] = U[i] + a1 * d[i];
        or_densities(p, Ut, pt, NULL, NULL);
        double h1 = 0.0;
        for (int64_t i = 0; i < n; ++i) h1 += (phi_target[i] - pt[i]) * d[i];
        double den = h1 - h0;
        double a = (den > 0.0) ? a1 * (-h0) / den : a1;
        for (int64_t i = 0; i < n; ++i) U[i] += a * d[i];
        or_densities(p, U, phi_model, NULL, NULL);
        gmax = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            g[i] = phi_target[i] - phi_model[i];
            if (fabs(g[i]) > gmax) gmax = fabs(g[i]);
        }
        double gg_new = dotv(g, g, n);
        double beta = (gg > 0.0) ? gg_new / gg : 0.0;
        for (int64_t i = 0; i < n; ++i) d[i] = -g[i] + beta * d[i];
        gg = gg_new;
        if (info) {
            info[2 + 4 * k + 0] = a1;
            info[2 + 4 * k + 1] = a;
            info[2 + 4 * k + 2] = gg;
            info[2 + 4 * k + 3] = gmax;
        }
    }
    free(g); free(d); free(Ut); free(pt);
    return k;
}

/* ------------------------------------------------------------------------------------ */
/* Intrinsic chemical potential, Eq. 4, with equal bead volumes (Sec. 2, units):          */
/*   mu_I = -U_I + sum_J chi_IJ sigma[phi_J] + kappa (sum_J phi_J - 1)                   */
/* Reading: the interaction kernel eps_IJ(r) is the same Gaussian as the bond kernel, so  */
/* its lattice form is the sigma stencil, and eps_IJ / (k_B T v0) = chi_IJ (eps_II = 0).  */
/* ------------------------------------------------------------------------------------ */
void or_mu(const or_params* p, const double* U, const double* phi, double* mu) {
    const int64_t V = nsites(p);
    const int ns = p->ns;
    double* sphi = (double*)malloc(sizeof(double) * (size_t)ns * (size_t)V);
    for (int J = 0; J < ns; ++J) or_sigma(p, phi + J * V, sphi + J * V);
    for (int64_t i = 0; i < V; ++i) {
        double tot = 0.0;
        for (int J = 0; J < ns; ++J) tot += phi[J * V + i];
        for (int I = 0; I < ns; ++I) {
            double m = -U[I * V + i];
            for (int J = 0; J < ns; ++J) m += p->chi[I * 3 + J] * sphi[J * V + i];
            m += p->kappa * (tot - 1.0);
            mu[I * V + i] = m;
        }
    }
    free(sphi);
}

/* Thermodynamic body force, Eq. 8: f = -sum_I phi_I grad mu_I, central differences. */
void or_force(const or_params* p, const double* phi, const double* mu, double* f) {
    const int64_t V = nsites(p);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                int64_t i = sidx(p, x, y, z);
                double fx = 0.0, fy = 0.0, fz = 0.0;
                for (int I = 0; I < p->ns; ++I) {
                    const double* m = mu + I * V;
                    double ph = phi[I * V + i];
                    fx -= ph * 0.5 * (m[sidx(p, x + 1, y, z)] - m[sidx(p, x - 1, y, z)]);
                    fy -= ph * 0.5 * (m[sidx(p, x, y + 1, z)] - m[sidx(p, x, y - 1, z)]);
                    fz -= ph * 0.5 * (m[sidx(p, x, y, z + 1)] - m[sidx(p, x, y, z - 1)]);
                }
                f[i] = fx; f[V + i] = fy; f[2 * V + i] = fz;
            }
}

/* ------------------------------------------------------------------------------------ */
/* Thermal noise (Sec. 2: Eq. 5 for the compositions, phi_k r_k in Eq. 13 for the LB).     */
/* Random numbers: Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and  */
/* Shaw (SC'11): ten rounds of two 32x32 -> 64-bit products of counter words with the      */
/* multipliers 0xD2511F53 and 0xCD9E8D57, the high halves XORed with the other two counter */
/* words and the key, the key bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85 between  */
/* rounds.  Key = (seed low 32 bits, seed high 32 bits).  Counter words (site, step,      */
/* stream, 0): stream 1 + I for the composition noise of species I, 16 + c (c = 0..3) for */
/* the LB modes.  Each output word gives a uniform u = (top 24 bits + 1/2) / 2^24 in       */
/* (0, 1); words (0, 1) and (2, 3) give two Box-Muller pairs                               */
/*   n = sqrt(-2 ln u_a) cos(2 pi u_b),  n' = sqrt(-2 ln u_a) sin(2 pi u_b).               */
/* ------------------------------------------------------------------------------------ */
void or_philox4x32(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* Four standard normals of counter (site, step, stream, 0). */
void or_normals4(uint64_t seed, uint32_t site, uint32_t step, uint32_t stream, double n[4]) {
    const uint32_t ctr[4] = {site, step, stream, 0u};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    or_philox4x32(ctr, key, r);
    double u[4];
    for (int i = 0; i < 4; ++i) u[i] = ((double)(r[i] >> 8) + 0.5) / 16777216.0;
    const double two_pi = 6.283185307179586476925286766559;
    for (int pr = 0; pr < 2; ++pr) {
        const double rad = sqrt(-2.0 * log(u[2 * pr]));
        n[2 * pr] = rad * cos(two_pi * u[2 * pr + 1]);
        n[2 * pr + 1] = rad * sin(two_pi * u[2 * pr + 1]);
    }
}

/* Composition noise of one step (Eq. 5), reading of the van Vlimmeren-Fraaije construction */
/* on the lattice: a random flux on every face, J_a(r) between r and r + e_a with variance   */
/* 2 M phi_face / (Omega dt) (phi_face the mean of the two sites, clipped at 0; the         */
/* 1/Omega = v0/h^3 turns bead densities into volume fractions), and the increment of the    */
/* step is minus its divergence,                                                              */
/*   dphi_I(r) = dt sum_a [J_a(r - e_a) - J_a(r)],                                            */
/* so its covariance is -(2/Omega) M dt div(phi grad delta) and every species' total is kept. */
/* J_a(r) = sqrt(2 M phi_face dt / Omega) n_a / dt with n_a the a-th normal of stream 1 + I.  */
void or_cd_noise(const or_params* p, const double* phi, double* dphi) {
    const int64_t V = nsites(p);
    const double amp2 = 2.0 * p->M * p->dt / p->omega;
    for (int I = 0; I < p->ns; ++I) {
        const double* ph = phi + I * V;
        double* J = (double*)malloc(sizeof(double) * 3 * (size_t)V);   /* dt * J_a(r), [a][V] */
#pragma omp parallel for schedule(static)
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    const int64_t i = sidx(p, x, y, z);
                    double n[4];
                    or_normals4(p->seed, (uint32_t)i, (uint32_t)p->step, 1u + (uint32_t)I, n);
                    const int64_t nb[3] = {sidx(p, x + 1, y, z), sidx(p, x, y + 1, z), sidx(p, x, y, z + 1)};
                    for (int a = 0; a < 3; ++a) {
                        double face = 0.5 * (ph[i] + ph[nb[a]]);
                        if (face < 0.0) face = 0.0;
                        J[a * V + i] = sqrt(amp2 * face) * n[a];
                    }
                }
#pragma omp parallel for schedule(static)
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    const int64_t i = sidx(p, x, y, z);
                    const int64_t lo[3] = {sidx(p, x - 1, y, z), sidx(p, x, y - 1, z), sidx(p, x, y, z - 1)};
                    double d = 0.0;
                    for (int a = 0; a < 3; ++a) d += J[a * V + lo[a]] - J[a * V + i];
                    dphi[I * V + i] = d;
                }
        free(J);
    }
}

/* ------------------------------------------------------------------------------------ */
/* D3Q19 multiple-relaxation-time lattice Boltzmann (Eq. 9-14, Table 1).                  */
/* ------------------------------------------------------------------------------------ */
static const int OR_C[19][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1}, {-1, 0, -1},
    {1, 0, -1}, {-1, 0, 1}, {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

/* Velocities, weights (text after Eq. 11), Table 1 eigenvectors (c = 1) and their norms   */
/* b_k = sum_i w_i e_ki^2 (text after Eq. 13).                                              */
void or_lb_basis(double e[19][19], double w[19], double b[19], int c[19][3]) {
    for (int i = 0; i < 19; ++i) {
        double cx = OR_C[i][0], cy = OR_C[i][1], cz = OR_C[i][2];
        double c2 = cx * cx + cy * cy + cz * cz;
        if (c) { c[i][0] = OR_C[i][0]; c[i][1] = OR_C[i][1]; c[i][2] = OR_C[i][2]; }
        w[i] = (c2 == 0.0) ? 1.0 / 3.0 : (c2 == 1.0 ? 1.0 / 18.0 : 1.0 / 36.0);
        e[0][i] = 1.0;
        e[1][i] = cx;
        e[2][i] = cy;
        e[3][i] = cz;
        e[4][i] = c2 - 1.0;
        e[5][i] = cx * cx - cy * cy;
        e[6][i] = c2 - 3.0 * cz * cz;
        e[7][i] = cx * cy;
        e[8][i] = cx * cz;
        e[9][i] = cy * cz;
        e[10][i] = (3.0 * c2 - 5.0) * cx;
        e[11][i] = (3.0 * c2 - 5.0) * cy;
        e[12][i] = (3.0 * c2 - 5.0) * cz;
        e[13][i] = (cy * cy - cz * cz) * cx;
        e[14][i] = (cz * cz - cx * cx) * cy;
        e[15][i] = (cx * cx - cy * cy) * cz;
        e[16][i] = 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
        e[17][i] = (2.0 * c2 - 3.0) * (cx * cx - cy * cy);
        e[18][i] = (2.0 * c2 - 3.0) * (c2 - 3.0 * cz * cz);
    }
    for (int k = 0; k < 19; ++k) {
        double s = 0.0;
        for (int i = 0; i < 19; ++i) s += w[i] * e[k][i] * e[k][i];
        b[k] = s;
    }
}

/* Second-order equilibrium, Eq. 11, with c_s^2 = 1/3 (lattice units). */
void or_lb_equilibrium(double rho, const double u[3], double neq[19]) {
    double e[19][19], w[19], b[19];
    int c[19][3];
    or_lb_basis(e, w, b, c);
    const double cs2 = 1.0 / 3.0;
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; ++i) {
        double uc = u[0] * c[i][0] + u[1] * c[i][1] + u[2] * c[i][2];
        neq[i] = rho * w[i] * (1.0 + uc / cs2 + 0.5 * uc * uc / (cs2 * cs2) - 0.5 * uu / cs2);
    }
}

/*
 * One LB step on the whole lattice: collision (Eq. 10, 12, 13 with phi_k = 0, force term
 * Eq. 14) followed by streaming n_i(r + c_i, t+1) = n*_i(r, t) (Eq. 10).
 *   n_in  [19][V]: populations n_i(r, t) before collision
 *   f     [3][V] : body force in lattice units (NULL = no force)
 *   n_out [19][V]: populations n_i(r, t+1) after streaming
 *   u_out [3][V] : velocity u = j/rho with j from Eq. 9 (half-force), NULL = not wanted
 */
void or_lb_step(const or_params* p, const double* n_in, const double* f, double* n_out, double* u_out) {
    const int64_t V = nsites(p);
    double e[19][19], w[19], b[19];
    int c[19][3];
    or_lb_basis(e, w, b, c);
    const double cs2 = 1.0 / 3.0;
    const double gs = 1.0 - 1.0 / p->tau_s;   /* relaxation parameter gamma_s */
    const double gb = 1.0 - 1.0 / p->tau_b;   /* relaxation parameter gamma_b */
    double gam[19];
    for (int k = 0; k < 19; ++k) gam[k] = (k <= 3) ? 1.0 : (k == 4 ? gb : (k <= 9 ? gs : 0.0));

#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                int64_t r = sidx(p, x, y, z);
                double n[19], fr[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < 19; ++i) n[i] = n_in[i * V + r];
                if (f) { fr[0] = f[r]; fr[1] = f[V + r]; fr[2] = f[2 * V + r]; }
                /* moments, Eq. 9 */
                double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < 19; ++i) {
                    rho += n[i];
                    for (int a = 0; a < 3; ++a) j[a] += n[i] * c[i][a];
                }
                double u[3];
                for (int a = 0; a < 3; ++a) { j[a] += 0.5 * fr[a]; u[a] = j[a] / rho; }
                if (u_out) { u_out[r] = u[0]; u_out[V + r] = u[1]; u_out[2 * V + r] = u[2]; }
                /* equilibrium, Eq. 11 */
                double neq[19];
                double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                for (int i = 0; i < 19; ++i) {
                    double uc = u[0] * c[i][0] + u[1] * c[i][1] + u[2] * c[i][2];
                    neq[i] = rho * w[i] * (1.0 + uc / cs2 + 0.5 * uc * uc / (cs2 * cs2) - 0.5 * uu / cs2);
                }
                /* forcing populations, Eq. 14 */
                double uf = u[0] * fr[0] + u[1] * fr[1] + u[2] * fr[2];
                double Sig[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int bb = 0; bb < 3; ++bb) {
                        double dab = (a == bb) ? 1.0 : 0.0;
                        Sig[a][bb] = 0.5 * (1.0 + gs) * (u[a] * fr[bb] + u[bb] * fr[a] - 2.0 / 3.0 * uf * dab)
                                   + 1.0 / 3.0 * (1.0 + gb) * uf * dab;
                    }
                double Df[19];
                for (int i = 0; i < 19; ++i) {
                    double fc = fr[0] * c[i][0] + fr[1] * c[i][1] + fr[2] * c[i][2];
                    double ss = 0.0;
                    for (int a = 0; a < 3; ++a)
                        for (int bb = 0; bb < 3; ++bb)
                            ss += Sig[a][bb] * (c[i][a] * c[i][bb] - cs2 * (a == bb ? 1.0 : 0.0));
                    Df[i] = w[i] / cs2 * (fc + 0.5 / cs2 * ss);
                }
                /* modes, Eq. 12; relaxation, Eq. 13; reconstruction */
                double ms[19];
                for (int k = 0; k < 19; ++k) {
                    double mk = 0.0, mf = 0.0;
                    for (int i = 0; i < 19; ++i) {
                        mk += (n[i] - neq[i]) * e[k][i];
                        mf += Df[i] * e[k][i];
                    }
                    ms[k] = gam[k] * mk + mf;
                }
                if (p->omega > 0.0 && p->lb_noise) {
                    /* phi_k r_k of Eq. 13 for the non-conserved modes k = 4..18, with the
                     * lattice-unit temperature kT = dt^2 / Omega (energy kT per bead, Omega
                     * beads of mass m0 per voxel, m0 = kT tau^2 / h^2) and c_s^2 = 1/3 */
                    const double kT = p->dt * p->dt / p->omega;
                    double g[16];
                    for (int cc = 0; cc < 4; ++cc)
                        or_normals4(p->seed, (uint32_t)r, (uint32_t)p->step, 16u + (uint32_t)cc, g + 4 * cc);
                    for (int k = 4; k < 19; ++k)
                        ms[k] += sqrt(rho * kT * b[k] * (1.0 - gam[k] * gam[k]) / cs2) * g[k - 4];
                }
                for (int i = 0; i < 19; ++i) {
                    double acc = 0.0;
                    for (int k = 0; k < 19; ++k) acc += ms[k] * e[k][i] / b[k];
                    double nstar = neq[i] + w[i] * acc;
                    /* streaming, Eq. 10 */
                    n_out[i * V + sidx(p, x + c[i][0], y + c[i][1], z + c[i][2])] = nstar;
                }
            }
}

/* ------------------------------------------------------------------------------------ */
/* Convection-diffusion update of the compositions, Eq. 3 (Sec. 2, finite-difference     */
/* paragraph: implicit Crank-Nicolson diffusion, explicit two-step Lax-Wendroff           */
/* convection).  Readings:                                                                */
/*  - convection: Richtmyer two-step Lax-Wendroff per axis in conservative form,          */
/*      phi_half(i+1/2) = (phi_i + phi_{i+1})/2 - (C_{i+1} phi_{i+1} - C_i phi_i)/2        */
/*      F(i+1/2)        = (C_i + C_{i+1})/2 * phi_half(i+1/2),   C = u_lat (Courant)       */
/*    and the axis fluxes are summed (unsplit);                                            */
/*  - diffusion: L(phi; mu)_i = sum_faces phi_face (mu_nb - mu_i), phi_face the mean of    */
/*    the two sites; Crank-Nicolson average of mu^n and mu^{n+1} with the mobility frozen  */
/*    at phi^n and mu^{n+1} linearised with the local curvature                            */
/*      mu^{n+1}_I ~ mu^n_I + delta_I / phi_I + kappa sum_J delta_J                        */
/*    (the large-wavevector limit of d mu/d phi), which gives the linear system            */
/*      delta - (dt M / 2) L(phi; H delta) = -conv + dt M L(phi; mu^n);                    */
/*  - the system is solved with cn_sweeps Jacobi sweeps from delta = 0, each sweep solving */
/*    the per-site species block exactly (Sherman-Morrison for the kappa coupling);        */
/*  - the result phi + delta is shifted per species to the prescribed totals mass0         */
/*    (mass0 == NULL: no shift).                                                          */
/* ------------------------------------------------------------------------------------ */
void or_cd_step(const or_params* p, const double* phi, const double* mu, const double* ulat,
                const double* mass0, double* phi_out) {
    const int64_t V = nsites(p);
    const int ns = p->ns;
    const double c = 0.5 * p->dt * p->M;
    const double fl = p->phi_floor;
    double* r = (double*)malloc(sizeof(double) * (size_t)ns * (size_t)V);
    double* del = (double*)calloc((size_t)ns * (size_t)V, sizeof(double));
    double* deln = (double*)malloc(sizeof(double) * (size_t)ns * (size_t)V);

#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                int64_t i = sidx(p, x, y, z);
                for (int I = 0; I < ns; ++I) {
                    const double* ph = phi + I * V;
                    const double* m = mu + I * V;
                    double conv = 0.0, lap = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        int ex = (d == 0), ey = (d == 1), ez = (d == 2);
                        int64_t ip = sidx(p, x + ex, y + ey, z + ez);
                        int64_t im = sidx(p, x - ex, y - ey, z - ez);
                        const double* C = ulat ? ulat + d * V : NULL;
                        double Ci = C ? C[i] : 0.0, Cp = C ? C[ip] : 0.0, Cm = C ? C[im] : 0.0;
                        /* face i+1/2 */
                        double hp = 0.5 * (ph[i] + ph[ip]) - 0.5 * (Cp * ph[ip] - Ci * ph[i]);
                        double Fp = 0.5 * (Ci + Cp) * hp;
                        /* face i-1/2 */
                        double hm = 0.5 * (ph[im] + ph[i]) - 0.5 * (Ci * ph[i] - Cm * ph[im]);
                        double Fm = 0.5 * (Cm + Ci) * hm;
                        conv += Fp - Fm;
                        lap += 0.5 * (ph[i] + ph[ip]) * (m[ip] - m[i]) + 0.5 * (ph[i] + ph[im]) * (m[im] - m[i]);
                    }
                    r[I * V + i] = -conv + p->dt * p->M * lap;
                }
            }
    if (p->omega > 0.0) {   /* thermal noise of the step enters the explicit part */
        double* dn = (double*)malloc(sizeof(double) * (size_t)ns * (size_t)V);
        or_cd_noise(p, phi, dn);
        for (int64_t k = 0; k < (int64_t)ns * V; ++k) r[k] += dn[k];
        free(dn);
    }

    for (int sweep = 0; sweep < p->cn_sweeps; ++sweep) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    int64_t i = sidx(p, x, y, z);
                    int64_t nb[6];
                    nb[0] = sidx(p, x + 1, y, z); nb[1] = sidx(p, x - 1, y, z);
                    nb[2] = sidx(p, x, y + 1, z); nb[3] = sidx(p, x, y - 1, z);
                    nb[4] = sidx(p, x, y, z + 1); nb[5] = sidx(p, x, y, z - 1);
                    /* psi at the neighbours from the previous iterate */
                    double psi[3][6];
                    for (int k = 0; k < 6; ++k) {
                        double sd = 0.0;
                        for (int J = 0; J < ns; ++J) sd += del[J * V + nb[k]];
                        for (int I = 0; I < ns; ++I) {
                            double ph = phi[I * V + nb[k]];
                            if (ph < fl) ph = fl;
                            psi[I][k] = del[I * V + nb[k]] / ph + p->kappa * sd;
                        }
                    }
                    double rhs[3], D[3], A[3];
                    for (int I = 0; I < ns; ++I) {
                        const double* ph = phi + I * V;
                        double wsum = 0.0, off = 0.0;
                        for (int k = 0; k < 6; ++k) {
                            double pf = 0.5 * (ph[i] + ph[nb[k]]);
                            wsum += pf;
                            off += pf * psi[I][k];
                        }
                        double phc = ph[i] < fl ? fl : ph[i];
                        rhs[I] = r[I * V + i] + c * off;
                        D[I] = 1.0 + c * wsum / phc;
                        A[I] = c * p->kappa * wsum;
                    }
                    /* (diag(D) + A 1^T) delta = rhs */
                    double num = 0.0, den = 1.0;
                    for (int I = 0; I < ns; ++I) { num += rhs[I] / D[I]; den += A[I] / D[I]; }
                    double s = num / den;
                    for (int I = 0; I < ns; ++I) deln[I * V + i] = (rhs[I] - A[I] * s) / D[I];
                }
        double* t = del; del = deln; deln = t;
    }

    for (int I = 0; I < ns; ++I) {
        double tot = 0.0;
        for (int64_t i = 0; i < V; ++i) {
            phi_out[I * V + i] = phi[I * V + i] + del[I * V + i];
            tot += phi_out[I * V + i];
        }
        double shift = mass0 ? (mass0[I] - tot) / (double)V : 0.0;
        for (int64_t i = 0; i < V; ++i) phi_out[I * V + i] += shift;
    }
    free(r); free(del); free(deln);
}

/* ------------------------------------------------------------------------------------ */
/* Starting point of the inversion (the paper does not say where the Fletcher-Reeves      */
/* iteration starts; reading: from the previous step's potentials, or with warm_extrap    */
/* from their linear extrapolation in time, 2 U^{n-1} - U^{n-2}, once two steps have      */
/* produced potentials).  Uprev holds U^{n-2} on entry and U^{n-1} on return.             */
/* ------------------------------------------------------------------------------------ */
void or_extrapolate(const or_params* p, double* U, double* Uprev) {
    const int64_t n = (int64_t)p->ns * nsites(p);
    for (int64_t i = 0; i < n; ++i) {
        const double u = U[i];
        U[i] = 2.0 * u - Uprev[i];
        Uprev[i] = u;
    }
}

/* ------------------------------------------------------------------------------------ */
/* One coupled time step (Sec. 2, paragraph after Eq. 17: LB steps alternate with         */
/* propagations of Eq. 3, each needing the self-consistent potentials).  Reading of the   */
/* order within a step:                                                                   */
/*   1. U^n  <- Fletcher-Reeves inversion of phi^n (warm start from the incoming U)       */
/*   2. mu^n <- Eq. 4                                                                      */
/*   3. if hydro: f = dt^2 * Eq. 8 (lattice units); LB step -> populations at n+1, u^n    */
/*   4. phi^{n+1} <- convection-diffusion with (phi^n, mu^n, u^n)                         */
/* State in/out: phi [ns][V] (replaced by phi^{n+1}), U [ns][V] (replaced by U^n),         */
/* pop [19][V] (post-streaming populations, replaced by those of step n+1; unused if     */
/* hydro == 0).  Outputs: mu [ns][V], ulat [3][V] (zero if hydro == 0), phim [ns][V] =    */
/* phi[U^n], info as in or_ncg.  With p->warm_extrap and Uprev != NULL the inversion starts */
/* from the extrapolated potentials (or_extrapolate).                                     */
/* ------------------------------------------------------------------------------------ */
void or_step(const or_params* p, double* phi, double* U, double* pop, const double* mass0,
             double* mu, double* ulat, double* phim, double* info, double* Uprev) {
    const int64_t V = nsites(p);
    const int ns = p->ns;
    if (p->warm_extrap && Uprev) or_extrapolate(p, U, Uprev);
    or_ncg(p, phi, U, phim, info);
    or_mu(p, U, phi, mu);
    if (p->hydro) {
        double* f = (double*)malloc(sizeof(double) * 3 * (size_t)V);
        double* pn = (double*)malloc(sizeof(double) * 19 * (size_t)V);
        or_force(p, phi, mu, f);
        for (int64_t i = 0; i < 3 * V; ++i) f[i] *= p->dt * p->dt;
        or_lb_step(p, pop, f, pn, ulat);
        memcpy(pop, pn, sizeof(double) * 19 * (size_t)V);
        free(f); free(pn);
    } else {
        for (int64_t i = 0; i < 3 * V; ++i) ulat[i] = 0.0;
    }
    double* pn = (double*)malloc(sizeof(double) * (size_t)ns * (size_t)V);
    or_cd_step(p, phi, mu, ulat, mass0, pn);
    memcpy(phi, pn, sizeof(double) * (size_t)ns * (size_t)V);
    free(pn);
}

/* ------------------------------------------------------------------------------------ */
/* Minkowski functionals of a thresholded field (Sec. 3, morphology of the aggregates;    */
/* the algorithm of Michielsen and De Raedt for a union of lattice cubes).  The body is   */
/* the union of the closed unit cubes at the sites where field > threshold (periodic      */
/* box).  Counting the distinct cubes n_c, faces n_f, edges n_e and vertices n_v of that   */
/* union,                                                                                  */
/*   V = n_c,  S = -6 n_c + 2 n_f,  2B = 3 n_c - 2 n_f + n_e,  chi = -n_c + n_f - n_e + n_v */
/* (volume, surface area, twice the integral mean curvature over pi in the lattice        */
/* normalisation, Euler characteristic of the body; a closed surface's own Euler number is */
/* 2 chi).  A face, edge or vertex belongs to the union when one of the 2, 4 or 8 cubes    */
/* that share it does; each is identified by the lattice point at its lower corner and an  */
/* orientation.  counts = {n_c, n_f, n_e, n_v}.                                           */
/* ------------------------------------------------------------------------------------ */
void or_minkowski_counts(int nx, int ny, int nz, const double* field, double threshold, int64_t counts[4]) {
    or_params p;
    memset(&p, 0, sizeof p);
    p.nx = nx; p.ny = ny; p.nz = nz;
    int64_t nc = 0, nf = 0, ne = 0, nv = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                /* in[dx][dy][dz]: the cube at (x - dx, y - dy, z - dz) is in the body */
                int in[2][2][2];
                for (int dx = 0; dx < 2; ++dx)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dz = 0; dz < 2; ++dz)
                            in[dx][dy][dz] = field[sidx(&p, x - dx, y - dy, z - dz)] > threshold;
                nc += in[0][0][0];
                /* faces at this lattice point, normal to x, y, z: shared with the cube below */
                nf += in[0][0][0] || in[1][0][0];
                nf += in[0][0][0] || in[0][1][0];
                nf += in[0][0][0] || in[0][0][1];
                /* edges from this lattice point along z, y, x: the four cubes around each */
                ne += in[0][0][0] || in[1][0][0] || in[0][1][0] || in[1][1][0];
                ne += in[0][0][0] || in[1][0][0] || in[0][0][1] || in[1][0][1];
                ne += in[0][0][0] || in[0][1][0] || in[0][0][1] || in[0][1][1];
                /* the vertex at this lattice point: the eight cubes around it */
                int any = 0;
                for (int dx = 0; dx < 2; ++dx)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dz = 0; dz < 2; ++dz) any |= in[dx][dy][dz];
                nv += any;
            }
    counts[0] = nc; counts[1] = nf; counts[2] = ne; counts[3] = nv;
}

/* ------------------------------------------------------------------------------------ */
/* Trapped solvent (Sec. 3: the solvent inside the vesicles, interior bulk solvent plus the */
/* hydration solvent of the inner leaflets, as a fraction of all solvent).  Reading: the   */
/* aggregates are the body {phi_B > threshold} (the hydrophobic cores, as for the         */
/* Minkowski functionals); its complement splits into face-connected components of the     */
/* periodic lattice; the largest is the bulk solvent outside, every other one is enclosed.  */
/* f_trap = sum of phi_S over the enclosed components / sum of phi_S over the box.         */
/* Components by breadth-first search; ties for the largest go to the one found first      */
/* (lowest site index).  Returns f_trap; *ncomp receives the number of complement         */
/* components.                                                                             */
/* ------------------------------------------------------------------------------------ */
double or_trapped_solvent(int nx, int ny, int nz, const double* phiB, const double* phiS, double threshold,
                          int64_t* ncomp) {
    or_params p;
    memset(&p, 0, sizeof p);
    p.nx = nx; p.ny = ny; p.nz = nz;
    const int64_t V = (int64_t)nx * ny * nz;
    int64_t* comp = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
    int64_t nc = 0, best = -1, best_size = -1;
    for (int64_t i = 0; i < V; ++i) comp[i] = (phiB[i] > threshold) ? -2 : -1;   /* -2 body, -1 unvisited */
    int64_t* sizes = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
    for (int64_t s0 = 0; s0 < V; ++s0) {
        if (comp[s0] != -1) continue;
        int64_t head = 0, tail = 0, size = 0;
        queue[tail++] = s0;
        comp[s0] = nc;
        while (head < tail) {
            const int64_t i = queue[head++];
            ++size;
            const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
            const int64_t nb[6] = {sidx(&p, x + 1, y, z), sidx(&p, x - 1, y, z), sidx(&p, x, y + 1, z),
                                   sidx(&p, x, y - 1, z), sidx(&p, x, y, z + 1), sidx(&p, x, y, z - 1)};
            for (int k = 0; k < 6; ++k)
                if (comp[nb[k]] == -1) { comp[nb[k]] = nc; queue[tail++] = nb[k]; }
        }
        sizes[nc] = size;
        if (size > best_size) { best_size = size; best = nc; }
        ++nc;
    }
    double trapped = 0.0, total = 0.0;
    for (int64_t i = 0; i < V; ++i) {
        total += phiS[i];
        if (comp[i] >= 0 && comp[i] != best) trapped += phiS[i];
    }
    if (ncomp) *ncomp = nc;
    free(comp); free(queue); free(sizes);
    return total > 0.0 ? trapped / total : 0.0;
}

/* ------------------------------------------------------------------------------------ */
/* Diagnostics.                                                                          */
/* Free-energy density v0 F/(k_B T V) of Eq. 1 in volume fractions (constants ln n!,      */
/* ln V and Omega dropped):                                                               */
/*   -(phi_p/N) ln Q - phi_s ln<exp(-U_S)> - V^-1 sum U_I phi_I                            */
/*   + (2V)^-1 sum sum_IJ chi_IJ phi_I sigma[phi_J] + kappa/(2V) sum (sum_I phi_I - 1)^2   */
/* ------------------------------------------------------------------------------------ */
double or_free_energy(const or_params* p, const double* U, const double* phi) {
    const int64_t V = nsites(p);
    const int ns = p->ns;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)ns * (size_t)V);
    double qs = 1.0;
    double Q = or_densities(p, U, tmp, &qs, NULL);
    double* sphi = tmp; /* reuse */
    double F = -p->phi_p / (double)p->N * log(Q);
    if (ns == 3) F -= (1.0 - p->phi_p) * log(qs);
    double acc = 0.0;
    for (int64_t i = 0; i < (int64_t)ns * V; ++i) acc += U[i] * phi[i];
    F -= acc / (double)V;
    double inter = 0.0;
    for (int J = 0; J < ns; ++J) {
        or_sigma(p, phi + J * V, sphi + J * V);
    }
    for (int64_t i = 0; i < V; ++i) {
        for (int I = 0; I < ns; ++I)
            for (int J = 0; J < ns; ++J) inter += 0.5 * p->chi[I * 3 + J] * phi[I * V + i] * sphi[J * V + i];
        double tot = -1.0;
        for (int I = 0; I < ns; ++I) tot += phi[I * V + i];
        inter += 0.5 * p->kappa * tot * tot;
    }
    F += inter / (double)V;
    free(tmp);
    return F;
}

/* Order parameter S of Fig. 1: sqrt(V^-1 sum_r sum_I (phi_I - <phi_I>)^2). */
double or_order_parameter(const or_params* p, const double* phi) {
    const int64_t V = nsites(p);
    double s2 = 0.0;
    for (int I = 0; I < p->ns; ++I) {
        double m = 0.0;
        for (int64_t i = 0; i < V; ++i) m += phi[I * V + i];
        m /= (double)V;
        for (int64_t i = 0; i < V; ++i) { double d = phi[I * V + i] - m; s2 += d * d; }
    }
    return sqrt(s2 / (double)V);
}

/* Segregation parameter of Fig. 3: V^-1 sum_r |phi_A + phi_B - <phi_A> - <phi_B>|. */
double or_segregation(const or_params* p, const double* phi) {
    const int64_t V = nsites(p);
    double mA = 0.0, mB = 0.0;
    for (int64_t i = 0; i < V; ++i) { mA += phi[i]; mB += phi[V + i]; }
    mA /= (double)V; mB /= (double)V;
    double s = 0.0;
    for (int64_t i = 0; i < V; ++i) s += fabs(phi[i] + phi[V + i] - mA - mB);
    return s / (double)V;
}

int or_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* Learned predictor (a small translation-invariant 3-D convolution network standing in  */
/* for the density map phi[U]; not part of the paper, see the package for its use).       */
/* Circular 3-D correlation with a 5^3 kernel centred on the site:                        */
/*   out[co][r] = b[co] + sum_ci sum_{o in [-2,2]^3} W[co][ci][o] in[ci][r + o]           */
/* W is [cout][cin][125] with offset index (oz+2)*25 + (oy+2)*5 + (ox+2); fields are     */
/* [c][V] for each of `batch` samples (sample-major), each sample periodic on its own.    */
/* ------------------------------------------------------------------------------------ */
void or_conv3d(int nx, int ny, int nz, int batch, int cin, int cout, const double* W, const double* b,
               const double* in, double* out) {
    const int64_t V = (int64_t)nx * ny * nz;
    for (int n = 0; n < batch; ++n) {
        const double* inn = in + (int64_t)n * cin * V;
        double* outn = out + (int64_t)n * cout * V;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const int64_t r = x + (int64_t)nx * (y + (int64_t)ny * z);
                    for (int co = 0; co < cout; ++co) {
                        double acc = b ? b[co] : 0.0;
                        for (int ci = 0; ci < cin; ++ci)
                            for (int oz = -2; oz <= 2; ++oz)
                                for (int oy = -2; oy <= 2; ++oy)
                                    for (int ox = -2; ox <= 2; ++ox) {
                                        const int o = (oz + 2) * 25 + (oy + 2) * 5 + (ox + 2);
                                        const int xs = ((x + ox) % nx + nx) % nx;
                                        const int ys = ((y + oy) % ny + ny) % ny;
                                        const int zs = ((z + oz) % nz + nz) % nz;
                                        acc += W[((int64_t)co * cin + ci) * 125 + o] *
                                               inn[(int64_t)ci * V + xs + (int64_t)nx * (ys + (int64_t)ny * zs)];
                                    }
                        outn[(int64_t)co * V + r] = acc;
                    }
                }
    }
}

/* Gradients of or_conv3d for an upstream gradient dout: dW (summed over sites and samples),
 * db, and din (NULL = not wanted):
 *   dW[co][ci][o] = sum_n sum_r dout[co][r] in[ci][r + o],  db[co] = sum_n sum_r dout[co][r],
 *   din[ci][r] = sum_co sum_o W[co][ci][o] dout[co][r - o]. */
void or_conv3d_bwd(int nx, int ny, int nz, int batch, int cin, int cout, const double* W, const double* in,
                   const double* dout, double* dW, double* db, double* din) {
    const int64_t V = (int64_t)nx * ny * nz;
    for (int64_t i = 0; i < (int64_t)cout * cin * 125; ++i) dW[i] = 0.0;
    for (int co = 0; co < cout; ++co) db[co] = 0.0;
    for (int n = 0; n < batch; ++n) {
        const double* inn = in + (int64_t)n * cin * V;
        const double* dn = dout + (int64_t)n * cout * V;
        for (int co = 0; co < cout; ++co)
            for (int64_t r = 0; r < V; ++r) db[co] += dn[(int64_t)co * V + r];
#pragma omp parallel for schedule(static)
        for (int co = 0; co < cout; ++co)
            for (int ci = 0; ci < cin; ++ci)
                for (int oz = -2; oz <= 2; ++oz)
                    for (int oy = -2; oy <= 2; ++oy)
                        for (int ox = -2; ox <= 2; ++ox) {
                            const int o = (oz + 2) * 25 + (oy + 2) * 5 + (ox + 2);
                            double acc = 0.0;
                            for (int z = 0; z < nz; ++z)
                                for (int y = 0; y < ny; ++y)
                                    for (int x = 0; x < nx; ++x) {
                                        const int xs = ((x + ox) % nx + nx) % nx;
                                        const int ys = ((y + oy) % ny + ny) % ny;
                                        const int zs = ((z + oz) % nz + nz) % nz;
                                        acc += dn[(int64_t)co * V + x + (int64_t)nx * (y + (int64_t)ny * z)] *
                                               inn[(int64_t)ci * V + xs + (int64_t)nx * (ys + (int64_t)ny * zs)];
                                    }
                            dW[((int64_t)co * cin + ci) * 125 + o] += acc;
                        }
        if (din) {
            double* dinn = din + (int64_t)n * cin * V;
#pragma omp parallel for schedule(static)
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x) {
                        for (int ci = 0; ci < cin; ++ci) {
                            double acc = 0.0;
                            for (int co = 0; co < cout; ++co)
                                for (int oz = -2; oz <= 2; ++oz)
                                    for (int oy = -2; oy <= 2; ++oy)
                                        for (int ox = -2; ox <= 2; ++ox) {
                                            const int o = (oz + 2) * 25 + (oy + 2) * 5 + (ox + 2);
                                            const int xs = ((x - ox) % nx + nx) % nx;
                                            const int ys = ((y - oy) % ny + ny) % ny;
                                            const int zs = ((z - oz) % nz + nz) % nz;
                                            acc += W[((int64_t)co * cin + ci) * 125 + o] *
                                                   dn[(int64_t)co * V + xs + (int64_t)nx * (ys + (int64_t)ny * zs)];
                                        }
                            dinn[(int64_t)ci * V + x + (int64_t)nx * (y + (int64_t)ny * z)] = acc;
                        }
                    }
        }
    }
}
