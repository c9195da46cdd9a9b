/*
 * FP64 CPU oracle for the lattice Boltzmann add-ons of Brownlee, Levesley,
 * Packwood and Gorban, "Add-ons for Lattice Boltzmann Methods:
 * Regularization, Filtering and Limiters".
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain, single-threaded
 * definition that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Layout of every population array: natural (pre-collision, post-stream)
 * state, structure of arrays f[i][y][x], i.e. index (i*ny + y)*nx + x, dense.
 *
 * D1Q3 velocities (Section 6):  i = 0,1,2  ->  v = -1, 0, +1.
 * D2Q9 velocities (Section 5, the paper's numbering 1..9 shifted to 0..8):
 *   0 rest, 1 E, 2 SE, 3 S, 4 SW, 5 W, 6 NW, 7 N, 8 NE   (y points north).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_D1Q3 = 1, ORC_D2Q9 = 2 };
enum { ORC_LBGK = 0, ORC_ELBM = 1, ORC_EHRENFEST = 2, ORC_POSITIVITY = 3,
       ORC_MEDIAN = 4, ORC_MRT = 5,
       /* limiters of Section 4.2-4.3, each f -> f* + phi(Delta S) (f - f*)
        * before the LBGK collision */
       ORC_SMOOTH = 6,            /* phi = 1 / (1 + alpha Delta S^k), Eq. smoothReg */
       ORC_DOUBLE_MONOTONIC = 7,  /* phi = (1 + (Delta S / Delta S_t)^k)^(-1/(2k)), Eq. DoublMonSpec */
       ORC_ENSEMBLE = 8,          /* Eq. phiExamp with the lattice mean E(Delta S) */
       ORC_THRESHOLD = 9,         /* Eqs. EntThresh, entrHom */
       /* Section 5's "aggressive" MRT A_2 = M_2^-1 C_2 M_2 */
       ORC_MRT2 = 10,             /* A_2 collision at every site (D2Q9) */
       ORC_MRT_LIMITER = 11,      /* LBGK, A_2 at the Ehrenfest-selected sites */
       /* Eq. phiExamp with E the mean of the PREVIOUS step's Delta S (the
        * first step of a call uses its own) */
       ORC_ENSEMBLE_LAGGED = 12 };
enum { ORC_EQ_POLY_PRODUCT = 0, ORC_EQ_ENTROPIC = 1, ORC_EQ_POLY_STD = 2 };
enum { ORC_BC_CAVITY = 0, ORC_BC_ENDS = 1, ORC_BC_PERIODIC = 2,
       ORC_BC_CHANNEL = 3,
       /* Section 8's diffusive Maxwell walls (D2Q9): the edge sites are
        * wall sites, not collided; the top wall moves with lid_u */
       ORC_BC_DIFFUSIVE = 4 };
enum { ORC_NORM_ENTROPIC = 0, ORC_NORM_L1 = 1 };
enum { ORC_FALLBACK_POSITIVITY = 0, ORC_FALLBACK_EHRENFEST = 1 };

typedef struct {
    int lattice;       /* ORC_D1Q3 | ORC_D2Q9 */
    int nx, ny;        /* ny = 1 for D1Q3 */
    int collision;     /* ORC_LBGK ... ORC_MRT */
    int equilibrium;   /* used by every collision except ELBM (always entropic) */
    int bc;            /* ORC_BC_* */
    double beta;       /* over-relaxation coefficient of Eq. (CollisionIntegral) */
    double lid_u;      /* velocity (along +x) of the top wall, cavity/channel */
    int topk;          /* Ehrenfest: at most this many sites per step */
    double delta;      /* Ehrenfest / median threshold on Delta S */
    double s_e, s_eps, s_q;  /* MRT rates of C1; s_nu = 2*beta */
    double elbm_eps;   /* stopping tolerance of Eq. (ConvergenceTwo) */
    int elbm_max_iter;
    int elbm_norm;     /* ORC_NORM_* */
    int elbm_fallback; /* ORC_FALLBACK_* */
    double lim_alpha;  /* alpha of Eqs. smoothReg / phiExamp */
    double lim_k;      /* k of Eqs. smoothReg / phiExamp / DoublMonSpec */
    double lim_dst;    /* Delta S_t of Eq. DoublMonSpec */
    double lim_delta0; /* delta_0 of Eqs. LimEntLim / EntThresh */
} orc_config;

typedef struct {
    long long limited_sites;     /* Ehrenfest / median / positivity corrections */
    long long candidates;        /* sites with Delta S > delta */
    long long elbm_solved;       /* sites that ran the root finder */
    long long elbm_skipped;      /* Delta S < 1e-15: plain LBGK step */
    long long elbm_fallbacks;    /* no non-trivial root */
    long long elbm_iters_total;
    long long elbm_iters_max;
    long long elbm_corrected;    /* double Newton step taken */
} orc_stats;

int orc_q(int lattice);
/* velocity components (cx, cy per direction) and the weights W_i */
void orc_lattice(int lattice, int* cx, int* cy, double* W);
int orc_opposite(int lattice, int i);

/* 1D equilibria of Section 6, functions of one velocity component. */
void orc_eq1d_poly(double u, double phi[3]);
void orc_eq1d_entropic(double u, double phi[3]);
/* Equilibrium populations at one site for the given kind. */
void orc_equilibrium(int lattice, int kind, double rho, double ux, double uy,
                     double* feq);
void orc_moments(int lattice, const double* f, double* rho, double* ux,
                 double* uy);

/* g(x) = (1+x) ln(1+x) - x, evaluated without cancellation. */
double orc_gfun(double x);
/* Delta S = sum_i f_i ln(f_i / f*_i) (Kullback form, Eq. DelS), in the
 * cancellation-free form sum_i f*_i g((f_i - f*_i)/f*_i).  +inf when any
 * population is non-positive. */
double orc_delta_s(int Q, const double* f, const double* feq);
/* The same quantity written literally as sum_i f_i ln(f_i/f*_i). */
double orc_delta_s_direct(int Q, const double* f, const double* feq);
/* S(f) = -sum_i f_i ln(f_i / W_i), the perfect-mixture entropy. */
double orc_entropy(int lattice, const double* f);
/* The D1Q3 entropy exactly as printed in Eq. (ELBMEntropy). */
double orc_entropy_d1q3_paper(const double f[3]);

/* ELBM root finder of Section 3.3 for one site.  feq must be the entropic
 * equilibrium.  Returns 0: root found, 1: near-equilibrium skip (alpha = 2),
 * 2: no non-trivial root (fallback rule applied). */
int orc_elbm_alpha(const orc_config* cfg, const double* f, const double* feq,
                   double* alpha, int* iters, int* corrected);
/* S_f(alpha) = S(f + alpha (f* - f)) - S(f) and its first two derivatives. */
void orc_elbm_sf(int Q, const double* f, const double* feq, double alpha,
                 double* s0, double* s1, double* s2);

/* MRT: A = M^{-1} C M of Section 5 (Q x Q, row major). */
void orc_mrt_basis(int lattice, double* M);
void orc_mrt_matrix(const orc_config* cfg, double* A);
/* M_2 of Section 5: rows 1, v_x, v_y, v_x^2+v_y^2, v_x^2-v_y^2, v_x v_y,
 * v_x v_y^2, v_x^2 v_y, v_x^2 v_y^2 (the printed row order) evaluated at
 * the velocities in this oracle's numbering; and A_2 = M_2^-1 C_2 M_2 with
 * C_2 = diag(1, 1, 1, 1, s_nu, s_nu, 1, 1, 1), s_nu = 2 beta (D2Q9). */
void orc_mrt2_basis(double* M);
void orc_mrt2_matrix(const orc_config* cfg, double* A);

/* Collide one site without the nonlocal limiters.  mode: the collision;
 * for EHRENFEST/MEDIAN the caller passes phi (1 = plain LBGK). */
void orc_collide_site(const orc_config* cfg, const double* f, double* F,
                      orc_stats* st);

/* Global selection of the Ehrenfest regularisation: mask[x] = 1 for the
 * min(k, |C|) sites of C = {x : dS[x] > delta} ordered by (dS desc, x asc). */
long long orc_select_topk(const double* dS, long long n, int k, double delta,
                          unsigned char* mask);
/* Limiter functions phi(Delta S) of Section 4.2-4.3 (+inf -> 0). */
double orc_phi_smooth(double dS, double alpha, double k);
double orc_phi_double_monotonic(double dS, double dst, double k);
/* E: the lattice mean of Delta S; E <= 0 (every site at equilibrium) -> 1 */
double orc_phi_ensemble(double dS, double alpha, double k, double E);
/* Delta S_0 of Eq. EntThresh for the empirical distribution of the n values
 * dS (non-finite values are left out): the t >= 0 with
 * sum_x max(dS_x - t, 0) = delta0 (1 - (2 beta - 1)^2) sum_x dS_x
 * (0 when the right-hand side reaches the whole sum). */
double orc_threshold_dS0(const double* dS, long long n, double delta0, double beta);

/* Lower median of the clipped (2r+1)^d window of dS (r = 1). */
void orc_median_field(int lattice, int nx, int ny, int periodic_x,
                      int periodic_y, const double* dS, double* med);

void orc_init_equilibrium(const orc_config* cfg, const double* rho,
                          const double* ux, const double* uy, double* f);
void orc_macros(const orc_config* cfg, const double* f, double* rho,
                double* ux, double* uy);
void orc_delta_s_field(const orc_config* cfg, const double* f, double* dS);
/* Enstrophy of Section 8: the sum over sites of the vorticity squared,
 * divided by the number of sites, with the vorticity
 * w = d u_y / dx - d u_x / dy by central differences of the site velocities
 * (periodic directions wrap; at a wall edge the one-sided difference to the
 * neighbour inside).  0 for D1Q3. */
double orc_enstrophy(const orc_config* cfg, const double* f);
/* H = sum_x sum_i f_i ln(f_i / W_i)  (= -S summed over the lattice). */
double orc_total_h(const orc_config* cfg, const double* f);

/* Advance nsteps collide-then-stream steps in place.  Returns 0 on success,
 * -1 on an invalid configuration, -2 on allocation failure. */
int orc_step(const orc_config* cfg, double* f, int nsteps, orc_stats* st);

/* Section 8's diffusive Maxwell rule on the wall sites of f (bc
 * ORC_BC_DIFFUSIVE), in place: at a site of one wall with outward normal n,
 * the populations pointing into the fluid (v . n < 0) become
 * gamma f*_i(u_wall), gamma = sum_{v.n > 0} f_j / sum_{v.n < 0} f*_i(u_wall)
 * (f* at unit density, u_wall = (lid_u, 0) on the top wall, 0 elsewhere);
 * at a corner each population whose source lies outside the box takes the
 * value of its opposite (the rule with a single population is
 * bounce-back).  Applied to the pre-collision state at the start of each
 * step. */
void orc_diffusive_rule(const orc_config* cfg, double* f);

/* Pure streaming with the boundary rule (used by the oracle step). */
void orc_stream(const orc_config* cfg, const double* F, double* fnew);

/* Kinetic energy J = 1/2 sum_x rho |u|^2 of a state. */
double orc_kinetic_energy(const orc_config* cfg, const double* f);

/* Tape-based reverse-mode gradient of J(f_T) = 1/2 sum_x rho |u|^2 after
 * T steps from f0, for the LBGK, Ehrenfest, median-filter and positivity
 * collisions (no diffusive walls).  The selection of each step is held
 * fixed and the selected branch differentiated: F = f* at the Ehrenfest
 * sites; F = f* + (1 - 2 beta) sqrt(M / C) (f - f*) at the median's sites,
 * with C = Delta S of the site and M = Delta S of the window site holding
 * the lower median (ties by site index) both differentiated; F = f* +
 * f*_k / (f*_k - f_k) (f - f*) where the positivity rule binds at population
 * k.  Outputs J, dJ/df0 (same layout as f0), dJ/d lid_u and dJ/d beta.
 * Returns 0, -1 for an unsupported configuration, -2 on allocation
 * failure. */
int orc_adjoint_ke(const orc_config* cfg, const double* f0, int T, double* J, double* dJ_df0,
                   double* dJ_dU, double* dJ_dbeta);

#ifdef __cplusplus
}
#endif
#endif
