/*
 * FP64 CPU oracle for the lattice Boltzmann add-ons of Brownlee, Levesley,
 * Packwood and Gorban.  TEST INFRASTRUCTURE ONLY: loaded by the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark, never by the
 * product path.  Single-threaded, plain loops, double precision throughout.
 *
 * Every function cites the passage of the paper it follows.  Where the paper
 * is silent or ambiguous, the reading taken is stated at the point of use.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Lattices.  D1Q3: Section 6 (v = -1, 0, 1).  D2Q9: Section 5 numbering,   */
/* rest first, then east, then clockwise; the weights W are the values of   */
/* the product equilibrium at rest (4/9, 1/9, 1/36).                        */
/* ------------------------------------------------------------------------ */

static const int D1_CX[3] = {-1, 0, 1};
static const double D1_W[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};

/* paper numbering 1..9 -> 0..8:  rest, E, SE, S, SW, W, NW, N, NE */
static const int D2_CX[9] = {0, 1, 1, 0, -1, -1, -1, 0, 1};
static const int D2_CY[9] = {0, 0, -1, -1, -1, 0, 1, 1, 1};

int orc_q(int lattice) { return lattice == ORC_D1Q3 ? 3 : (lattice == ORC_D2Q9 ? 9 : 0); }

static double d2_weight(int i) {
    int s = D2_CX[i] * D2_CX[i] + D2_CY[i] * D2_CY[i];
    return s == 0 ? 4.0 / 9.0 : (s == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
}

void orc_lattice(int lattice, int* cx, int* cy, double* W) {
    int Q = orc_q(lattice);
    for (int i = 0; i < Q; ++i) {
        if (lattice == ORC_D1Q3) {
            cx[i] = D1_CX[i];
            cy[i] = 0;
            W[i] = D1_W[i];
        } else {
            cx[i] = D2_CX[i];
            cy[i] = D2_CY[i];
            W[i] = d2_weight(i);
        }
    }
}

/* The opposite direction is found by search: the velocity equal to -c_i. */
int orc_opposite(int lattice, int i) {
    int Q = orc_q(lattice);
    int cx[9], cy[9];
    double W[9];
    orc_lattice(lattice, cx, cy, W);
    for (int j = 0; j < Q; ++j)
        if (cx[j] == -cx[i] && cy[j] == -cy[i]) return j;
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Equilibria (Section 6 for D1Q3; Section 8 states that the D2Q9           */
/* quasi-equilibrium is the product of the 1D ones).                        */
/* ------------------------------------------------------------------------ */

/* Polynomial 1D equilibrium per unit density, order (-, 0, +). */
void orc_eq1d_poly(double u, double phi[3]) {
    phi[0] = (1.0 - 3.0 * u + 3.0 * u * u) / 6.0;
    phi[1] = 2.0 / 3.0 * (1.0 - 1.5 * u * u);
    phi[2] = (1.0 + 3.0 * u + 3.0 * u * u) / 6.0;
}

/* Entropic 1D equilibrium per unit density, order (-, 0, +). */
void orc_eq1d_entropic(double u, double phi[3]) {
    double s = sqrt(1.0 + 3.0 * u * u);
    phi[0] = (-3.0 * u - 1.0 + 2.0 * s) / 6.0;
    phi[1] = 2.0 / 3.0 * (2.0 - s);
    phi[2] = (3.0 * u - 1.0 + 2.0 * s) / 6.0;
}

void orc_equilibrium(int lattice, int kind, double rho, double ux, double uy,
                     double* feq) {
    double px[3], py[3];
    if (lattice == ORC_D1Q3) {
        if (kind == ORC_EQ_ENTROPIC)
            orc_eq1d_entropic(ux, px);
        else
            orc_eq1d_poly(ux, px);
        for (int i = 0; i < 3; ++i) feq[i] = rho * px[i];
        return;
    }
    if (kind == ORC_EQ_POLY_STD) {
        /* The textbook second-order polynomial, offered as an option:
         * W_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2). */
        double uu = ux * ux + uy * uy;
        for (int i = 0; i < 9; ++i) {
            double cu = D2_CX[i] * ux + D2_CY[i] * uy;
            feq[i] = d2_weight(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        }
        return;
    }
    if (kind == ORC_EQ_ENTROPIC) {
        orc_eq1d_entropic(ux, px);
        orc_eq1d_entropic(uy, py);
    } else {
        orc_eq1d_poly(ux, px);
        orc_eq1d_poly(uy, py);
    }
    /* phi index of velocity component c is c + 1 */
    for (int i = 0; i < 9; ++i) feq[i] = rho * px[D2_CX[i] + 1] * py[D2_CY[i] + 1];
}

/* {rho, rho u} = sum_i {1, v_i} f_i  (Section 2). */
void orc_moments(int lattice, const double* f, double* rho, double* ux, double* uy) {
    int Q = orc_q(lattice);
    int cx[9], cy[9];
    double W[9];
    orc_lattice(lattice, cx, cy, W);
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < Q; ++i) {
        r += f[i];
        jx += cx[i] * f[i];
        jy += cy[i] * f[i];
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
}

/* ------------------------------------------------------------------------ */
/* Entropies (Section 3.1, Eq. ELBMEntropy; Section 4, Eqs. Kul, DelS).     */
/* ------------------------------------------------------------------------ */

/* g(x) = (1+x) ln(1+x) - x.  For small |x| the closed form cancels, so the
 * Taylor series sum_{n>=2} (-1)^n x^n / (n (n-1)) is summed instead. */
double orc_gfun(double x) {
    if (x < -1.0) return NAN;
    if (x == -1.0) return 1.0;
    if (fabs(x) < 0.25) {
        double sum = 0.0, p = x * x;
        for (int n = 2; n < 80; ++n) {
            double term = p / ((double)n * (double)(n - 1));
            sum += (n % 2 == 0) ? term : -term;
            if (fabs(term) < 1e-19 * fabs(sum)) break;
            p *= x;
        }
        return sum;
    }
    return (1.0 + x) * log1p(x) - x;
}

/* Nonequilibrium entropy Delta S = sum f ln(f/f*) (Eq. DelS).  Since every
 * equilibrium used here carries the same density as f, adding
 * sum (f* - f) = 0 turns each term into f*_i g(x_i), x_i = (f_i - f*_i)/f*_i,
 * which is free of cancellation.  Reading: a negative population makes the
 * logarithm undefined; Delta S is then +inf (the site is as far from
 * equilibrium as it gets). */
double orc_delta_s(int Q, const double* f, const double* feq) {
    double s = 0.0;
    for (int i = 0; i < Q; ++i) {
        if (f[i] < 0.0 || !(feq[i] > 0.0)) return INFINITY;
        s += feq[i] * orc_gfun((f[i] - feq[i]) / feq[i]);
    }
    return s;
}

double orc_delta_s_direct(int Q, const double* f, const double* feq) {
    double s = 0.0;
    for (int i = 0; i < Q; ++i) {
        if (f[i] < 0.0 || !(feq[i] > 0.0)) return INFINITY;
        if (f[i] > 0.0) s += f[i] * log(f[i] / feq[i]);
    }
    return s;
}

double orc_entropy(int lattice, const double* f) {
    int Q = orc_q(lattice);
    int cx[9], cy[9];
    double W[9];
    orc_lattice(lattice, cx, cy, W);
    double s = 0.0;
    for (int i = 0; i < Q; ++i)
        if (f[i] > 0.0) s -= f[i] * log(f[i] / W[i]);
    return s;
}

double orc_entropy_d1q3_paper(const double f[3]) {
    return -f[0] * log(f[0]) - f[1] * log(f[1] / 4.0) - f[2] * log(f[2]);
}

/* ------------------------------------------------------------------------ */
/* ELBM (Section 3).                                                        */
/* ------------------------------------------------------------------------ */

/* S_f(alpha) = S(f + alpha Delta) - S(f), Delta = f* - f (Eq. NewCondition),
 * with its derivatives in alpha.  For an entropic equilibrium,
 * S(y) = S(f*) - DeltaS(y) for every y with the moments of f* (the Lagrange
 * form of ln f* in Section 4), so S_f(alpha) = DeltaS(f) - DeltaS(g),
 * g = f + alpha Delta.  Writing d_i = Delta_i / f*_i, the relative
 * deviation of g is x_i = (alpha - 1) d_i and
 *   S_f   = sum f*_i [ g(-d_i) - g(x_i) ],
 *   S_f'  = -sum Delta_i ln(1 + x_i),
 *   S_f'' = -sum Delta_i^2 / g_i.                                          */
void orc_elbm_sf(int Q, const double* f, const double* feq, double alpha,
                 double* s0, double* s1, double* s2) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = 0; i < Q; ++i) {
        double D = feq[i] - f[i];
        double d = D / feq[i];
        double x = (alpha - 1.0) * d;
        if (x < -1.0) x = -1.0; /* g_i = 0 at the positivity limit */
        a += feq[i] * (orc_gfun(-d) - orc_gfun(x));
        b -= D * log1p(x);
        c -= D * D / (f[i] + alpha * D);
    }
    *s0 = a;
    *s1 = b;
    *s2 = c;
}

static double elbm_norm(const orc_config* cfg, int Q, const double* f, const double* feq) {
    double n = 0.0;
    for (int i = 0; i < Q; ++i) {
        double D = feq[i] - f[i];
        if (cfg->elbm_norm == ORC_NORM_L1)
            n += fabs(D);
        else
            n += D * D / feq[i];
    }
    /* Reading: the entropic norm is printed as the quadratic form itself; a
     * norm must be homogeneous of degree one, so its square root is used. */
    return cfg->elbm_norm == ORC_NORM_L1 ? n : sqrt(n);
}

/* Root finder of Section 3.3:
 *  - sites with Delta S < 1e-15 take the LBGK step (alpha = 2);
 *  - start at the LBGK estimate alpha_0 = 2;
 *  - each iterate is the greater root of the second-order Taylor parabola
 *    of S_f at the current estimate;
 *  - stop when |S_f / S_f'| * ||f* - f|| < eps (Eqs. Stopping, ConvergenceTwo);
 *  - if S_f < 0 at the stop, take the double-length Newton step back.
 * Readings where the paper is silent:
 *  - the admissible interval is (1, alpha_max], alpha_max the largest alpha
 *    with f + alpha Delta >= 0 (S_f(1) = Delta S > 0 always).  If 2 is not
 *    admissible the start is the midpoint of (1, alpha_max);
 *  - when S_f > 0 at the start, existence of a non-trivial root is decided
 *    by the sign of S_f(alpha_max); without one, the rule of Section 3.2
 *    chosen by cfg->elbm_fallback applies (positivity: alpha = alpha_max;
 *    Ehrenfest: alpha = 1);
 *  - a parabola root outside the current bracket, or a negative
 *    discriminant, is replaced by the bracket midpoint. */
int orc_elbm_alpha(const orc_config* cfg, const double* f, const double* feq,
                   double* alpha, int* iters, int* corrected) {
    int Q = orc_q(cfg->lattice);
    *iters = 0;
    *corrected = 0;
    double dS = orc_delta_s(Q, f, feq);
    if (dS < 1e-15) {
        *alpha = 2.0;
        return 1;
    }
    double amax = INFINITY;
    int negative = 0;
    for (int i = 0; i < Q; ++i) {
        double D = feq[i] - f[i];
        if (f[i] < 0.0) negative = 1;
        if (D < 0.0) {
            double a = -f[i] / D;
            if (a < amax) amax = a;
        }
    }
    double fallback = cfg->elbm_fallback == ORC_FALLBACK_EHRENFEST ? 1.0 : amax;
    if (negative) { /* S(f) undefined: no entropy condition to solve */
        *alpha = fallback;
        return 2;
    }
    double nrm = elbm_norm(cfg, Q, f, feq);
    double lo = 1.0, hi = amax;
    double a = (2.0 < amax) ? 2.0 : 0.5 * (1.0 + amax);
    double s0, s1, s2;
    orc_elbm_sf(Q, f, feq, a, &s0, &s1, &s2);
    if (s0 > 0.0) {
        double m0, m1, m2;
        orc_elbm_sf(Q, f, feq, amax, &m0, &m1, &m2);
        if (m0 > 0.0) {
            *alpha = fallback;
            return 2;
        }
        lo = a;
    } else {
        hi = a;
    }
    int it = 0;
    while (it < cfg->elbm_max_iter) {
        if (fabs(s0 / s1) * nrm < cfg->elbm_eps) break;
        ++it;
        double disc = s1 * s1 - 2.0 * s0 * s2;
        double next = NAN;
        if (disc >= 0.0) {
            double r1 = (-s1 + sqrt(disc)) / s2;
            double r2 = (-s1 - sqrt(disc)) / s2;
            next = a + (r1 > r2 ? r1 : r2);
        }
        if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
        a = next;
        orc_elbm_sf(Q, f, feq, a, &s0, &s1, &s2);
        if (s0 > 0.0)
            lo = a;
        else
            hi = a;
    }
    if (s0 < 0.0) {
        a = a - 2.0 * s0 / s1;
        *corrected = 1;
    }
    *iters = it;
    *alpha = a;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* MRT (Section 5).                                                         */
/* ------------------------------------------------------------------------ */

/* D2Q9 basis M1 of Section 5 in the paper's velocity numbering; D1Q3 uses
 * the monomials {1, v, v^2} (the paper has no D1Q3 MRT). */
void orc_mrt_basis(int lattice, double* M) {
    static const int M1[9][9] = {
        {1, 1, 1, 1, 1, 1, 1, 1, 1},
        {-4, -1, 2, -1, 2, -1, 2, -1, 2},
        {4, -2, 1, -2, 1, -2, 1, -2, 1},
        {0, 1, 1, 0, -1, -1, -1, 0, 1},
        {0, -2, 1, 0, -1, 2, -1, 0, 1},
        {0, 0, -1, -1, -1, 0, 1, 1, 1},
        {0, 0, -1, 2, -1, 0, 1, -2, 1},
        {0, 1, 0, -1, 0, 1, 0, -1, 0},
        {0, 0, -1, 0, 1, 0, -1, 0, 1}};
    if (lattice == ORC_D2Q9) {
        for (int r = 0; r < 9; ++r)
            for (int c = 0; c < 9; ++c) M[r * 9 + c] = M1[r][c];
    } else {
        for (int i = 0; i < 3; ++i) {
            double v = D1_CX[i];
            M[0 * 3 + i] = 1.0;
            M[1 * 3 + i] = v;
            M[2 * 3 + i] = v * v;
        }
    }
}

/* Gauss-Jordan inversion with partial pivoting (plain, n <= 9). */
static int invert(int n, const double* A, double* inv) {
    double a[9][18];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            a[r][c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = t;
            }
        double p = a[col][col];
        for (int c = 0; c < 2 * n; ++c) a[col][c] /= p;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            for (int c = 0; c < 2 * n; ++c) a[r][c] -= m * a[col][c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) inv[r * n + c] = a[r][c + n];
    return 0;
}

/* A1 = M1^{-1} C1 M1 with C1 = diag(1, s_e, s_eps, 1, s_q, 1, s_q, s_nu, s_nu)
 * and s_nu = 2 beta (so that equal rates reproduce LBGK's 2 beta).  D1Q3:
 * C = diag(1, 1, s_nu). */
void orc_mrt_matrix(const orc_config* cfg, double* A) {
    int Q = orc_q(cfg->lattice);
    double M[81], Minv[81], C[9];
    double snu = 2.0 * cfg->beta;
    orc_mrt_basis(cfg->lattice, M);
    invert(Q, M, Minv);
    if (Q == 9) {
        double c9[9] = {1.0, cfg->s_e, cfg->s_eps, 1.0, cfg->s_q, 1.0, cfg->s_q, snu, snu};
        memcpy(C, c9, sizeof c9);
    } else {
        C[0] = 1.0;
        C[1] = 1.0;
        C[2] = snu;
    }
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < Q; ++c) {
            double s = 0.0;
            for (int k = 0; k < Q; ++k) s += Minv[r * Q + k] * C[k] * M[k * Q + c];
            A[r * Q + c] = s;
        }
}

void orc_mrt2_basis(double* M) {
    int cx[9], cy[9];
    double W[9];
    orc_lattice(ORC_D2Q9, cx, cy, W);
    for (int i = 0; i < 9; ++i) {
        double x = cx[i], y = cy[i];
        double row[9] = {1.0, x, y, x * x + y * y, x * x - y * y, x * y, x * y * y, x * x * y, x * x * y * y};
        for (int r = 0; r < 9; ++r) M[r * 9 + i] = row[r];
    }
}

void orc_mrt2_matrix(const orc_config* cfg, double* A) {
    double M[81], Minv[81];
    double snu = 2.0 * cfg->beta;
    double C[9] = {1.0, 1.0, 1.0, 1.0, snu, snu, 1.0, 1.0, 1.0};
    orc_mrt2_basis(M);
    invert(9, M, Minv);
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
            double s = 0.0;
            for (int k = 0; k < 9; ++k) s += Minv[r * 9 + k] * C[k] * M[k * 9 + c];
            A[r * 9 + c] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* Collisions.                                                              */
/* ------------------------------------------------------------------------ */

static int eq_kind(const orc_config* cfg) {
    return cfg->collision == ORC_ELBM ? ORC_EQ_ENTROPIC : cfg->equilibrium;
}

static void site_equilibrium(const orc_config* cfg, const double* f, double* feq) {
    double rho, ux, uy;
    orc_moments(cfg->lattice, f, &rho, &ux, &uy);
    orc_equilibrium(cfg->lattice, eq_kind(cfg), rho, ux, uy, feq);
}

/* LBGK with over-relaxation, Eq. (CollisionIntegral) with alpha = 2. */
static void lbgk(int Q, double beta, const double* f, const double* feq, double* F) {
    for (int i = 0; i < Q; ++i) F[i] = f[i] + 2.0 * beta * (feq[i] - f[i]);
}

/* Positivity rule (Section 4, Eq. StrLine): a state with a negative
 * component is replaced by the nonnegative point of the line through it and
 * f* closest to it, F = f* + lambda (F - f*),
 * lambda = min over F_i < 0 of f*_i / (f*_i - F_i). */
static int positivity(int Q, const double* feq, double* F) {
    double lam = 1.0;
    int hit = 0;
    for (int i = 0; i < Q; ++i)
        if (F[i] < 0.0) {
            double l = feq[i] / (feq[i] - F[i]);
            if (l < lam) lam = l;
            hit = 1;
        }
    if (!hit) return 0;
    for (int i = 0; i < Q; ++i) F[i] = feq[i] + lam * (F[i] - feq[i]);
    return 1;
}

static void collide_local(const orc_config* cfg, const double* A, const double* f,
                          double* F, orc_stats* st) {
    int Q = orc_q(cfg->lattice);
    double feq[9];
    site_equilibrium(cfg, f, feq);
    switch (cfg->collision) {
        case ORC_ELBM: {
            double alpha;
            int iters, corr;
            int rc = orc_elbm_alpha(cfg, f, feq, &alpha, &iters, &corr);
            if (st) {
                if (rc == 1) st->elbm_skipped++;
                if (rc == 2) st->elbm_fallbacks++;
                if (rc == 0) st->elbm_solved++;
                st->elbm_iters_total += iters;
                if (iters > st->elbm_iters_max) st->elbm_iters_max = iters;
                st->elbm_corrected += corr;
            }
            for (int i = 0; i < Q; ++i) F[i] = f[i] + alpha * cfg->beta * (feq[i] - f[i]);
            break;
        }
        case ORC_MRT:
        case ORC_MRT2: {
            /* A holds A_1 or A_2 (the caller's choice by collision) */
            for (int r = 0; r < Q; ++r) {
                double s = 0.0;
                for (int c = 0; c < Q; ++c) s += A[r * Q + c] * (feq[c] - f[c]);
                F[r] = f[r] + s;
            }
            break;
        }
        case ORC_POSITIVITY:
            lbgk(Q, cfg->beta, f, feq, F);
            if (positivity(Q, feq, F) && st) st->limited_sites++;
            break;
        default:
            lbgk(Q, cfg->beta, f, feq, F);
            break;
    }
}

void orc_collide_site(const orc_config* cfg, const double* f, double* F, orc_stats* st) {
    double A[81];
    if (cfg->collision == ORC_MRT) orc_mrt_matrix(cfg, A);
    if (cfg->collision == ORC_MRT2) orc_mrt2_matrix(cfg, A);
    collide_local(cfg, A, f, F, st);
}

/* ------------------------------------------------------------------------ */
/* Nonlocal limiters (Section 4).                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    double ds;
    long long idx;
} cand_t;

static int cand_cmp(const void* pa, const void* pb) {
    const cand_t* a = (const cand_t*)pa;
    const cand_t* b = (const cand_t*)pb;
    if (a->ds > b->ds) return -1;
    if (a->ds < b->ds) return 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

/* Ehrenfest regularisation (Section 4): among the sites whose Delta S
 * exceeds delta, the k with the largest Delta S.  Reading: ties are broken
 * by the lower site index; fewer than k candidates are all taken. */
long long orc_select_topk(const double* dS, long long n, int k, double delta,
                          unsigned char* mask) {
    long long nc = 0;
    for (long long x = 0; x < n; ++x) {
        mask[x] = 0;
        if (dS[x] > delta) ++nc;
    }
    if (nc == 0 || k <= 0) return nc;
    cand_t* c = (cand_t*)malloc(sizeof(cand_t) * (size_t)nc);
    if (!c) return -1;
    long long m = 0;
    for (long long x = 0; x < n; ++x)
        if (dS[x] > delta) {
            c[m].ds = dS[x];
            c[m].idx = x;
            ++m;
        }
    qsort(c, (size_t)nc, sizeof(cand_t), cand_cmp);
    long long take = nc < k ? nc : k;
    for (long long j = 0; j < take; ++j) mask[c[j].idx] = 1;
    free(c);
    return nc;
}

static int dbl_cmp(const void* pa, const void* pb) {
    double a = *(const double*)pa, b = *(const double*)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Median entropy filter (Section 4.4): the median of Delta S over the site
 * and its nearest neighbours (3 in 1D, 9 in 2D).  Reading: at a wall the
 * window is clipped to the sites that exist and the lower median (element
 * floor((n-1)/2) of the ascending order) is taken; periodic directions wrap. */
void orc_median_field(int lattice, int nx, int ny, int periodic_x, int periodic_y,
                      const double* dS, double* med) {
    int ry = lattice == ORC_D2Q9 ? 1 : 0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double w[9];
            int n = 0;
            for (int dy = -ry; dy <= ry; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int xx = x + dx, yy = y + dy;
                    if (periodic_x) xx = (xx + nx) % nx;
                    if (periodic_y) yy = (yy + ny) % ny;
                    if (xx < 0 || xx >= nx || yy < 0 || yy >= ny) continue;
                    w[n++] = dS[(long long)yy * nx + xx];
                }
            qsort(w, (size_t)n, sizeof(double), dbl_cmp);
            med[(long long)y * nx + x] = w[(n - 1) / 2];
        }
}

/* ------------------------------------------------------------------------ */
/* Streaming and boundaries.                                                */
/* ------------------------------------------------------------------------ */

static void bc_periodicity(const orc_config* cfg, int* px, int* py) {
    *px = (cfg->bc == ORC_BC_PERIODIC || cfg->bc == ORC_BC_CHANNEL);
    *py = (cfg->bc == ORC_BC_PERIODIC);
}

/* Advection f_i(x + v_i) <- F_i(x) (Section 2).  A population whose target
 * lies outside the domain is bounced back half-way into the opposite
 * direction at its own site (Section 8's bounce-back).  Crossing the top
 * wall, which moves with velocity (lid_u, 0), adds the moving-wall term
 * -6 W_i rho_w (v_i . u_wall) with rho_w = 1; links through the two top
 * corners count as lid links. */
void orc_stream(const orc_config* cfg, const double* F, double* fnew) {
    int Q = orc_q(cfg->lattice);
    int nx = cfg->nx, ny = cfg->ny;
    long long N = (long long)nx * ny;
    int cx[9], cy[9];
    double W[9];
    orc_lattice(cfg->lattice, cx, cy, W);
    int px, py;
    bc_periodicity(cfg, &px, &py);
    for (int i = 0; i < Q; ++i) {
        int o = orc_opposite(cfg->lattice, i);
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double v = F[i * N + (long long)y * nx + x];
                int tx = x + cx[i], ty = y + cy[i];
                if (px) tx = (tx + nx) % nx;
                if (py) ty = (ty + ny) % ny;
                if (tx >= 0 && tx < nx && ty >= 0 && ty < ny) {
                    fnew[i * N + (long long)ty * nx + tx] = v;
                } else {
                    double corr = 0.0;
                    if (ty >= ny && cfg->bc != ORC_BC_DIFFUSIVE) corr = 6.0 * W[i] * 1.0 * (cx[i] * cfg->lid_u);
                    fnew[o * N + (long long)y * nx + x] = v - corr;
                }
            }
    }
}

void orc_diffusive_rule(const orc_config* cfg, double* f) {
    if (cfg->bc != ORC_BC_DIFFUSIVE || cfg->lattice != ORC_D2Q9) return;
    int nx = cfg->nx, ny = cfg->ny;
    long long N = (long long)nx * ny;
    int cx[9], cy[9];
    double W[9];
    orc_lattice(ORC_D2Q9, cx, cy, W);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int nxw = (x == 0 ? -1 : 0) + (x == nx - 1 ? 1 : 0);
            int nyw = (y == 0 ? -1 : 0) + (y == ny - 1 ? 1 : 0);
            if (nxw == 0 && nyw == 0) continue; /* a fluid site */
            long long s = (long long)y * nx + x;
            if (nxw != 0 && nyw != 0) {
                /* corner: bounce-back for the populations from outside */
                double fs[9];
                for (int i = 0; i < 9; ++i) fs[i] = f[i * N + s];
                for (int i = 0; i < 9; ++i) {
                    int sx = x - cx[i], sy = y - cy[i];
                    if (sx < 0 || sx >= nx || sy < 0 || sy >= ny) {
                        int o = orc_opposite(ORC_D2Q9, i);
                        int ox = x - cx[o], oy = y - cy[o];
                        if (ox >= 0 && ox < nx && oy >= 0 && oy < ny) f[i * N + s] = fs[o];
                    }
                }
                continue;
            }
            double uw = (nyw == 1) ? cfg->lid_u : 0.0;
            double feq[9];
            orc_equilibrium(ORC_D2Q9, eq_kind(cfg), 1.0, uw, 0.0, feq);
            double out = 0.0, in = 0.0;
            for (int i = 0; i < 9; ++i) {
                int vn = cx[i] * nxw + cy[i] * nyw;
                if (vn > 0) out += f[i * N + s];
                if (vn < 0) in += feq[i];
            }
            double gamma = out / in;
            for (int i = 0; i < 9; ++i)
                if (cx[i] * nxw + cy[i] * nyw < 0) f[i * N + s] = gamma * feq[i];
        }
}

static int is_wall_site(const orc_config* cfg, long long s) {
    if (cfg->bc != ORC_BC_DIFFUSIVE) return 0;
    int x = (int)(s % cfg->nx), y = (int)(s / cfg->nx);
    return x == 0 || x == cfg->nx - 1 || y == 0 || y == cfg->ny - 1;
}

/* ------------------------------------------------------------------------ */
/* Fields and the full step.                                                */
/* ------------------------------------------------------------------------ */

static void gather(int Q, const double* f, long long N, long long s, double* out) {
    for (int i = 0; i < Q; ++i) out[i] = f[i * N + s];
}

void orc_init_equilibrium(const orc_config* cfg, const double* rho, const double* ux,
                          const double* uy, double* f) {
    int Q = orc_q(cfg->lattice);
    long long N = (long long)cfg->nx * cfg->ny;
    double feq[9];
    for (long long s = 0; s < N; ++s) {
        orc_equilibrium(cfg->lattice, eq_kind(cfg), rho[s], ux[s], uy ? uy[s] : 0.0, feq);
        for (int i = 0; i < Q; ++i) f[i * N + s] = feq[i];
    }
}

void orc_macros(const orc_config* cfg, const double* f, double* rho, double* ux, double* uy) {
    int Q = orc_q(cfg->lattice);
    long long N = (long long)cfg->nx * cfg->ny;
    double fs[9];
    for (long long s = 0; s < N; ++s) {
        double r, a, b;
        gather(Q, f, N, s, fs);
        orc_moments(cfg->lattice, fs, &r, &a, &b);
        rho[s] = r;
        ux[s] = a;
        if (uy) uy[s] = b;
    }
}

void orc_delta_s_field(const orc_config* cfg, const double* f, double* dS) {
    int Q = orc_q(cfg->lattice);
    long long N = (long long)cfg->nx * cfg->ny;
    double fs[9], feq[9];
    for (long long s = 0; s < N; ++s) {
        gather(Q, f, N, s, fs);
        site_equilibrium(cfg, fs, feq);
        dS[s] = orc_delta_s(Q, fs, feq);
    }
}

double orc_total_h(const orc_config* cfg, const double* f) {
    int Q = orc_q(cfg->lattice);
    long long N = (long long)cfg->nx * cfg->ny;
    double fs[9], h = 0.0;
    for (long long s = 0; s < N; ++s) {
        gather(Q, f, N, s, fs);
        h -= orc_entropy(cfg->lattice, fs);
    }
    return h;
}

/* d g / d coordinate at index i of a line of n values with spacing 1. */
static double diff1(const double* g, long long stride, int i, int n, int periodic) {
    if (n < 2) return 0.0;
    if (periodic) {
        int ip = i + 1 < n ? i + 1 : 0, im = i > 0 ? i - 1 : n - 1;
        return 0.5 * (g[ip * stride] - g[im * stride]);
    }
    if (i == 0) return g[1 * stride] - g[0];
    if (i == n - 1) return g[(long long)i * stride] - g[(long long)(i - 1) * stride];
    return 0.5 * (g[(long long)(i + 1) * stride] - g[(long long)(i - 1) * stride]);
}

double orc_enstrophy(const orc_config* cfg, const double* f) {
    if (cfg->lattice != ORC_D2Q9) return 0.0;
    int nx = cfg->nx, ny = cfg->ny, px, py;
    long long N = (long long)nx * ny;
    bc_periodicity(cfg, &px, &py);
    double* rho = (double*)malloc(sizeof(double) * (size_t)N);
    double* ux = (double*)malloc(sizeof(double) * (size_t)N);
    double* uy = (double*)malloc(sizeof(double) * (size_t)N);
    if (!rho || !ux || !uy) {
        free(rho);
        free(ux);
        free(uy);
        return -1.0;
    }
    orc_macros(cfg, f, rho, ux, uy);
    double e = 0.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            /* d u_y / dx along the row, d u_x / dy along the column */
            double dvdx = diff1(uy + (long long)y * nx + 0, 1, x, nx, px);
            double dudy = diff1(ux + x, nx, y, ny, py);
            double w = dvdx - dudy;
            e += w * w;
        }
    free(rho);
    free(ux);
    free(uy);
    return e / (double)N;
}

static int config_ok(const orc_config* cfg) {
    if (cfg->lattice != ORC_D1Q3 && cfg->lattice != ORC_D2Q9) return 0;
    if (cfg->nx < 1 || cfg->ny < 1) return 0;
    if (cfg->lattice == ORC_D1Q3 && cfg->ny != 1) return 0;
    if (cfg->collision < ORC_LBGK || cfg->collision > ORC_ENSEMBLE_LAGGED) return 0;
    if ((cfg->collision == ORC_MRT2 || cfg->collision == ORC_MRT_LIMITER) && cfg->lattice != ORC_D2Q9) return 0;
    if (cfg->bc == ORC_BC_DIFFUSIVE && (cfg->lattice != ORC_D2Q9 || cfg->nx < 3 || cfg->ny < 3)) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Limiter functions of Section 4.2 (smooth regularisation, Eq. smoothReg;  */
/* ensemble-dependent phi, Eq. phiExamp), Section 4.3 (double monotonic,    */
/* Eq. DoublMonSpec) and Section 4.4 (threshold, Eqs. EntThresh, entrHom).  */
/* A state with Delta S = +inf (a negative population) goes to f*: each phi */
/* tends to 0 as Delta S grows.                                              */
/* ------------------------------------------------------------------------ */

double orc_phi_smooth(double dS, double alpha, double k) {
    if (isinf(dS)) return 0.0;
    return 1.0 / (1.0 + alpha * pow(dS, k));
}

double orc_phi_double_monotonic(double dS, double dst, double k) {
    if (isinf(dS)) return 0.0;
    return pow(1.0 + pow(dS / dst, k), -1.0 / (2.0 * k));
}

double orc_phi_ensemble(double dS, double alpha, double k, double E) {
    if (isinf(dS)) return 0.0;
    if (!(E > 0.0)) return 1.0;
    double y = dS / (alpha * E);
    return (1.0 + pow(y, k - 0.5)) / (1.0 + pow(y, k));
}

static int cmp_desc(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return x < y ? 1 : (x > y ? -1 : 0);
}

double orc_threshold_dS0(const double* dS, long long n, double delta0, double beta) {
    /* finite values, sorted in decreasing order */
    double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!v) return -1.0;
    long long m = 0;
    double total = 0.0;
    for (long long x = 0; x < n; ++x)
        if (isfinite(dS[x])) {
            v[m++] = dS[x];
            total += dS[x];
        }
    qsort(v, (size_t)m, sizeof(double), cmp_desc);
    double c = 1.0 - (2.0 * beta - 1.0) * (2.0 * beta - 1.0);
    double R = delta0 * c * total;
    /* L(t) = sum_x max(v_x - t, 0) is continuous, piecewise linear and
     * decreasing; on [v_(j+1), v_(j)] (j values above) it is
     * S_j - j t with S_j the sum of the j largest values.  Walk down the
     * sorted values until L at the next one reaches R. */
    double t = 0.0, S = 0.0;
    int found = 0;
    for (long long j = 1; j <= m; ++j) {
        S += v[j - 1];
        double next = j < m ? v[j] : 0.0;      /* lower end of the piece */
        double Lnext = S - (double)j * next;   /* L(next) */
        if (Lnext >= R) {
            t = (S - R) / (double)j;           /* solve S_j - j t = R */
            found = 1;
            break;
        }
    }
    if (!found) t = 0.0;  /* R >= L(0): every value is above the threshold */
    free(v);
    return t < 0.0 ? 0.0 : t;
}

/* One step of Section 2's scheme, collide then stream, applied nsteps times.
 * The nonequilibrium entropy field of every site is computed from the
 * pre-collision state before any site is collided (reading: the paper does
 * not order these; a Jacobi sweep makes the result independent of site
 * order). */
int orc_step(const orc_config* cfg, double* f, int nsteps, orc_stats* st) {
    if (!config_ok(cfg)) return -1;
    int Q = orc_q(cfg->lattice);
    long long N = (long long)cfg->nx * cfg->ny;
    double* F = (double*)malloc(sizeof(double) * (size_t)(Q * N));
    double* dS = (double*)malloc(sizeof(double) * (size_t)N);
    double* med = (double*)malloc(sizeof(double) * (size_t)N);
    unsigned char* mask = (unsigned char*)malloc((size_t)N);
    if (!F || !dS || !med || !mask) {
        free(F);
        free(dS);
        free(med);
        free(mask);
        return -2;
    }
    int px, py;
    bc_periodicity(cfg, &px, &py);
    double A[81];
    if (cfg->collision == ORC_MRT) orc_mrt_matrix(cfg, A);
    if (cfg->collision == ORC_MRT2 || cfg->collision == ORC_MRT_LIMITER) orc_mrt2_matrix(cfg, A);
    int diffusive = cfg->bc == ORC_BC_DIFFUSIVE;
    double E_prev = 0.0; /* the lagged ensemble limiter's E of the previous step */
    for (int t = 0; t < nsteps; ++t) {
        double fs[9], feq[9], Fs[9];
        if (diffusive) orc_diffusive_rule(cfg, f);
        int nonlocal = cfg->collision == ORC_EHRENFEST || cfg->collision == ORC_MEDIAN ||
                       (cfg->collision >= ORC_SMOOTH && cfg->collision != ORC_MRT2);
        double E = 0.0, dSt = 0.0;
        if (nonlocal) {
            orc_delta_s_field(cfg, f, dS);
            /* wall sites are not collided: never limiter candidates, and the
             * median windows are clipped to the fluid sites */
            if (diffusive)
                for (long long x = 0; x < N; ++x)
                    if (is_wall_site(cfg, x)) dS[x] = 0.0;
            if (cfg->collision == ORC_EHRENFEST || cfg->collision == ORC_MRT_LIMITER) {
                long long nc = orc_select_topk(dS, N, cfg->topk, cfg->delta, mask);
                if (st) st->candidates += nc;
            } else if (cfg->collision == ORC_MEDIAN && diffusive) {
                int ix = cfg->nx - 2, iy = cfg->ny - 2;
                double* sub = (double*)malloc(sizeof(double) * (size_t)ix * iy * 2);
                if (!sub) {
                    free(F);
                    free(dS);
                    free(med);
                    free(mask);
                    return -2;
                }
                for (int y = 0; y < iy; ++y)
                    for (int x = 0; x < ix; ++x) sub[(long long)y * ix + x] = dS[(long long)(y + 1) * cfg->nx + x + 1];
                orc_median_field(cfg->lattice, ix, iy, 0, 0, sub, sub + (long long)ix * iy);
                for (int y = 0; y < iy; ++y)
                    for (int x = 0; x < ix; ++x)
                        med[(long long)(y + 1) * cfg->nx + x + 1] = sub[(long long)ix * iy + (long long)y * ix + x];
                free(sub);
            } else if (cfg->collision == ORC_MEDIAN) {
                orc_median_field(cfg->lattice, cfg->nx, cfg->ny, px, py, dS, med);
            } else if (cfg->collision == ORC_ENSEMBLE || cfg->collision == ORC_ENSEMBLE_LAGGED) {
                /* E(Delta S): mean over the sites with a finite value */
                long long nf = 0;
                for (long long x = 0; x < N; ++x)
                    if (isfinite(dS[x]) && !is_wall_site(cfg, x)) {
                        E += dS[x];
                        ++nf;
                    }
                E = nf > 0 ? E / (double)nf : 0.0;
                if (cfg->collision == ORC_ENSEMBLE_LAGGED) {
                    /* reading: E of the previous step's pre-collision state,
                     * this step's own in the first step */
                    double E_now = E;
                    if (t > 0) E = E_prev;
                    E_prev = E_now;
                }
            } else if (cfg->collision == ORC_THRESHOLD) {
                /* Delta S_t = max(Delta S_0, delta) */
                double d0 = orc_threshold_dS0(dS, N, cfg->lim_delta0, cfg->beta);
                dSt = d0 > cfg->delta ? d0 : cfg->delta;
            }
        }
        for (long long s = 0; s < N; ++s) {
            gather(Q, f, N, s, fs);
            if (diffusive && is_wall_site(cfg, s)) {
                /* wall sites are not collided (Section 8) */
                for (int i = 0; i < Q; ++i) F[i * N + s] = fs[i];
                continue;
            }
            if (!nonlocal) {
                collide_local(cfg, A, fs, Fs, st);
            } else if (cfg->collision == ORC_MRT_LIMITER) {
                /* Section 5: the A_2 collision at the selected sites (the
                 * Ehrenfest selection of Section 4), LBGK elsewhere */
                site_equilibrium(cfg, fs, feq);
                if (mask[s]) {
                    for (int r = 0; r < Q; ++r) {
                        double acc = 0.0;
                        for (int c = 0; c < Q; ++c) acc += A[r * Q + c] * (feq[c] - fs[c]);
                        Fs[r] = fs[r] + acc;
                    }
                    if (st) st->limited_sites++;
                } else {
                    lbgk(Q, cfg->beta, fs, feq, Fs);
                }
            } else {
                site_equilibrium(cfg, fs, feq);
                double phi = 1.0;
                int limited = 0;
                if (cfg->collision == ORC_EHRENFEST) {
                    if (mask[s]) {
                        phi = 0.0; /* Ehrenfest step f -> f* */
                        limited = 1;
                    }
                } else if (cfg->collision == ORC_MEDIAN) {
                    /* median filter with the homothety of Eq. (entrHom),
                     * accepted only when it lowers Delta S */
                    if (st && dS[s] > cfg->delta) st->candidates++;
                    if (dS[s] > cfg->delta && med[s] < dS[s]) {
                        phi = isinf(dS[s]) ? 0.0 : sqrt(med[s] / dS[s]);
                        limited = 1;
                    }
                } else if (cfg->collision == ORC_THRESHOLD) {
                    /* homothety of Eq. (entrHom) where Delta S >= Delta S_t */
                    if (dS[s] >= dSt) {
                        phi = isinf(dS[s]) ? 0.0 : sqrt(dSt / dS[s]);
                        limited = 1;
                    }
                } else {
                    if (cfg->collision == ORC_SMOOTH)
                        phi = orc_phi_smooth(dS[s], cfg->lim_alpha, cfg->lim_k);
                    else if (cfg->collision == ORC_DOUBLE_MONOTONIC)
                        phi = orc_phi_double_monotonic(dS[s], cfg->lim_dst, cfg->lim_k);
                    else
                        phi = orc_phi_ensemble(dS[s], cfg->lim_alpha, cfg->lim_k, E);
                    limited = phi != 1.0;
                }
                /* limiter f -> f* + phi (f - f*) (Eq. LimGenF), then LBGK */
                for (int i = 0; i < Q; ++i) {
                    double fl = feq[i] + phi * (fs[i] - feq[i]);
                    Fs[i] = fl + 2.0 * cfg->beta * (feq[i] - fl);
                }
                if (st && limited) st->limited_sites++;
            }
            for (int i = 0; i < Q; ++i) F[i * N + s] = Fs[i];
        }
        orc_stream(cfg, F, f);
    }
    free(F);
    free(dS);
    free(med);
    free(mask);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reverse-mode gradient (adjoint) of the kinetic energy after T steps.     */
/* ------------------------------------------------------------------------ */

double orc_kinetic_energy(const orc_config* cfg, const double* f) {
    int Q = orc_q(cfg->lattice);
    long long N = (long long)cfg->nx * cfg->ny;
    double fs[9], e = 0.0;
    for (long long s = 0; s < N; ++s) {
        double r, ux, uy;
        gather(Q, f, N, s, fs);
        orc_moments(cfg->lattice, fs, &r, &ux, &uy);
        e += 0.5 * r * (ux * ux + uy * uy);
    }
    return e;
}

/* Derivatives of the 1D equilibria (per unit density) in u. */
static void eq1d_deriv(int kind, double u, double phi[3], double dphi[3]) {
    if (kind == ORC_EQ_ENTROPIC) {
        double s = sqrt(1.0 + 3.0 * u * u);
        orc_eq1d_entropic(u, phi);
        dphi[0] = -0.5 + u / s;
        dphi[1] = -2.0 * u / s;
        dphi[2] = 0.5 + u / s;
    } else {
        orc_eq1d_poly(u, phi);
        dphi[0] = u - 0.5;
        dphi[1] = -2.0 * u;
        dphi[2] = u + 0.5;
    }
}

/* df*_i/d(rho), d/d(ux), d/d(uy) at one site. */
static void eq_partials(int lattice, int kind, double rho, double ux, double uy, double* dr,
                        double* dx, double* dy) {
    int Q = orc_q(lattice);
    int cx[9], cy[9];
    double W[9];
    orc_lattice(lattice, cx, cy, W);
    if (lattice == ORC_D2Q9 && kind == ORC_EQ_POLY_STD) {
        double uu = ux * ux + uy * uy;
        for (int i = 0; i < Q; ++i) {
            double cu = cx[i] * ux + cy[i] * uy;
            dr[i] = W[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            dx[i] = W[i] * rho * (3.0 * cx[i] + 9.0 * cu * cx[i] - 3.0 * ux);
            dy[i] = W[i] * rho * (3.0 * cy[i] + 9.0 * cu * cy[i] - 3.0 * uy);
        }
        return;
    }
    double px[3], dpx[3], py[3] = {0.0, 1.0, 0.0}, dpy[3] = {0.0, 0.0, 0.0};
    eq1d_deriv(kind, ux, px, dpx);
    if (lattice == ORC_D2Q9) eq1d_deriv(kind, uy, py, dpy);
    for (int i = 0; i < Q; ++i) {
        int a = cx[i] + 1, b = cy[i] + 1;
        dr[i] = px[a] * py[b];
        dx[i] = rho * dpx[a] * py[b];
        dy[i] = rho * px[a] * dpy[b];
    }
}

/* Delta S at one site and its gradient dDelta S / df_j (Eq. DelS):
 * Delta S = sum_i f_i ln(f_i / f*_i(f)), so
 * dDelta S / df_j = ln(f_j / f*_j) + 1 - sum_i (f_i / f*_i) df*_i / df_j
 * with df*_i / df_j = df*_i/drho + df*_i/du_x (v_jx - u_x)/rho + df*_i/du_y (v_jy - u_y)/rho. */
static double delta_s_grad(const orc_config* cfg, const double* f, double* grad) {
    int Q = orc_q(cfg->lattice);
    int cx[9], cy[9];
    double W[9], feq[9], dr[9], dx[9], dy[9], r, ux, uy;
    orc_lattice(cfg->lattice, cx, cy, W);
    orc_moments(cfg->lattice, f, &r, &ux, &uy);
    orc_equilibrium(cfg->lattice, eq_kind(cfg), r, ux, uy, feq);
    eq_partials(cfg->lattice, eq_kind(cfg), r, ux, uy, dr, dx, dy);
    for (int j = 0; j < Q; ++j) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i)
            s += f[i] / feq[i] * (dr[i] + dx[i] * (cx[j] - ux) / r + dy[i] * (cy[j] - uy) / r);
        grad[j] = log(f[j] / feq[j]) + 1.0 - s;
    }
    return orc_delta_s(Q, f, feq);
}

/* The window site whose Delta S is the lower median of the clipped window
 * of site s (the value orc_median_field takes), with ties in Delta S
 * ordered by the site index. */
static long long median_site(const orc_config* cfg, int px, int py, const double* dS, long long s) {
    int ry = cfg->lattice == ORC_D2Q9 ? 1 : 0;
    int x = (int)(s % cfg->nx), y = (int)(s / cfg->nx);
    long long w[9];
    int n = 0;
    for (int dy = -ry; dy <= ry; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            int xx = x + dx, yy = y + dy;
            if (px) xx = (xx + cfg->nx) % cfg->nx;
            if (py) yy = (yy + cfg->ny) % cfg->ny;
            if (xx < 0 || xx >= cfg->nx || yy < 0 || yy >= cfg->ny) continue;
            long long v = (long long)yy * cfg->nx + xx;
            int k = n++;
            while (k > 0 && (dS[w[k - 1]] > dS[v] || (dS[w[k - 1]] == dS[v] && w[k - 1] > v))) {
                w[k] = w[k - 1];
                --k;
            }
            w[k] = v;
        }
    return w[(n - 1) / 2];
}

/* Branch codes of one site in one step of the tape (the selection that the
 * adjoint holds fixed); every branch has the form F = f* + psi (f - f*):
 *   AUX_LBGK          psi = 1 - 2 beta (Eq. CollisionIntegral)
 *   AUX_FSTAR         psi = 0 (the Ehrenfest step of Section 4)
 *   AUX_POS0 - k      the positivity rule of Eq. (StrLine) binding at
 *                     population k: psi = f*_k / (f*_k - f_k)
 *   m >= 0            the median filter of Section 4.4 with the window's
 *                     lower median at site m: psi = (1 - 2 beta) sqrt(Delta S(m) / Delta S) */
enum { AUX_LBGK = -1, AUX_FSTAR = -2, AUX_POS0 = -3 };

int orc_adjoint_ke(const orc_config* cfg, const double* f0, int T, double* J, double* dJ_df0,
                   double* dJ_dU, double* dJ_dbeta) {
    if (!config_ok(cfg) || T < 0) return -1;
    if (cfg->collision != ORC_LBGK && cfg->collision != ORC_EHRENFEST && cfg->collision != ORC_MEDIAN &&
        cfg->collision != ORC_POSITIVITY)
        return -1;
    if (cfg->bc == ORC_BC_DIFFUSIVE) return -1;
    int Q = orc_q(cfg->lattice);
    long long N = (long long)cfg->nx * cfg->ny;
    size_t S = (size_t)(Q * N);
    double* tape = (double*)malloc(sizeof(double) * S * (size_t)(T + 1));
    long long* aux = (long long*)malloc(sizeof(long long) * (size_t)N * (size_t)(T > 0 ? T : 1));
    unsigned char* mask = (unsigned char*)malloc((size_t)N);
    double* F = (double*)malloc(sizeof(double) * S);
    double* dS = (double*)malloc(sizeof(double) * (size_t)N);
    double* lam = (double*)malloc(sizeof(double) * S);
    double* Lam = (double*)malloc(sizeof(double) * S);
    if (!tape || !aux || !mask || !F || !dS || !lam || !Lam) {
        free(tape); free(aux); free(mask); free(F); free(dS); free(lam); free(Lam);
        return -2;
    }
    int cx[9], cy[9];
    double W[9];
    orc_lattice(cfg->lattice, cx, cy, W);
    int px, py;
    bc_periodicity(cfg, &px, &py);
    const int kind = eq_kind(cfg);
    const double c = 1.0 - 2.0 * cfg->beta;

    /* forward, keeping every pre-collision state and each site's branch */
    memcpy(tape, f0, sizeof(double) * S);
    for (int t = 0; t < T; ++t) {
        const double* f = tape + (size_t)t * S;
        long long* a = aux + (size_t)t * N;
        for (long long s = 0; s < N; ++s) a[s] = AUX_LBGK;
        if (cfg->collision == ORC_EHRENFEST || cfg->collision == ORC_MEDIAN) orc_delta_s_field(cfg, f, dS);
        if (cfg->collision == ORC_EHRENFEST) {
            orc_select_topk(dS, N, cfg->topk, cfg->delta, mask);
            for (long long s = 0; s < N; ++s)
                if (mask[s]) a[s] = AUX_FSTAR;
        }
        /* the same arithmetic as orc_step, branch by branch */
        for (long long s = 0; s < N; ++s) {
            double fs[9], feq[9], Fs[9];
            gather(Q, f, N, s, fs);
            site_equilibrium(cfg, fs, feq);
            if (cfg->collision == ORC_LBGK || cfg->collision == ORC_POSITIVITY) {
                lbgk(Q, cfg->beta, fs, feq, Fs);
                if (cfg->collision == ORC_POSITIVITY) {
                    /* the rule's binding population: the first i with the
                     * smallest f*_i / (f*_i - F_i) over F_i < 0 */
                    double lam_min = 1.0;
                    int k = -1;
                    for (int i = 0; i < Q; ++i)
                        if (Fs[i] < 0.0) {
                            double l = feq[i] / (feq[i] - Fs[i]);
                            if (l < lam_min) {
                                lam_min = l;
                                k = i;
                            }
                        }
                    if (k >= 0) {
                        a[s] = AUX_POS0 - k;
                        positivity(Q, feq, Fs);
                    }
                }
            } else {
                double phi = a[s] == AUX_FSTAR ? 0.0 : 1.0;
                if (cfg->collision == ORC_MEDIAN && dS[s] > cfg->delta) {
                    long long m = median_site(cfg, px, py, dS, s);
                    if (dS[m] < dS[s]) {
                        a[s] = m;
                        phi = isinf(dS[s]) ? 0.0 : sqrt(dS[m] / dS[s]);
                    }
                }
                for (int i = 0; i < Q; ++i) {
                    double fl = feq[i] + phi * (fs[i] - feq[i]);
                    Fs[i] = fl + 2.0 * cfg->beta * (feq[i] - fl);
                }
            }
            for (int i = 0; i < Q; ++i) F[i * N + s] = Fs[i];
        }
        orc_stream(cfg, F, tape + (size_t)(t + 1) * S);
    }
    const double* fT = tape + (size_t)T * S;
    *J = orc_kinetic_energy(cfg, fT);

    /* seed: dJ/df_j = c_j . u - |u|^2 / 2 at every site */
    for (long long s = 0; s < N; ++s) {
        double fs[9], r, ux, uy;
        gather(Q, fT, N, s, fs);
        orc_moments(cfg->lattice, fs, &r, &ux, &uy);
        for (int j = 0; j < Q; ++j)
            lam[j * N + s] = cx[j] * ux + cy[j] * uy - 0.5 * (ux * ux + uy * uy);
    }
    double gU = 0.0, gB = 0.0;
    for (int t = T - 1; t >= 0; --t) {
        /* transpose of the streaming: F_i(x) went to (i, x + v_i), or bounced
         * to (opp(i), x) with the moving-wall term -6 W_i v_ix U */
        for (int i = 0; i < Q; ++i) {
            int o = orc_opposite(cfg->lattice, i);
            for (int y = 0; y < cfg->ny; ++y)
                for (int x = 0; x < cfg->nx; ++x) {
                    int tx = x + cx[i], ty = y + cy[i];
                    if (px) tx = (tx + cfg->nx) % cfg->nx;
                    if (py) ty = (ty + cfg->ny) % cfg->ny;
                    long long s = (long long)y * cfg->nx + x;
                    if (tx >= 0 && tx < cfg->nx && ty >= 0 && ty < cfg->ny) {
                        Lam[i * N + s] = lam[i * N + (long long)ty * cfg->nx + tx];
                    } else {
                        Lam[i * N + s] = lam[o * N + s];
                        if (ty >= cfg->ny) gU += lam[o * N + s] * (-6.0 * W[i] * cx[i]);
                    }
                }
        }
        /* transpose of the collision F = f* + psi (f - f*) at every site:
         * dF_i/df_j = (1 - psi) df*_i/df_j + psi delta_ij + (f_i - f*_i) dpsi/df_j,
         * dF_i/dbeta = (f_i - f*_i) dpsi/dbeta; the median's psi also depends
         * on the state at its window site m (added there) */
        const double* f = tape + (size_t)t * S;
        const long long* a = aux + (size_t)t * N;
        for (long long s = 0; s < N; ++s) {
            double fs[9], feq[9], dr[9], dx[9], dy[9], r, ux, uy, L[9], dfk[9];
            gather(Q, f, N, s, fs);
            gather(Q, Lam, N, s, L);
            orc_moments(cfg->lattice, fs, &r, &ux, &uy);
            orc_equilibrium(cfg->lattice, kind, r, ux, uy, feq);
            eq_partials(cfg->lattice, kind, r, ux, uy, dr, dx, dy);
            /* a_j = sum_i L_i df*_i/df_j with drho/df_j = 1,
             * du_x/df_j = (v_jx - u_x)/rho, du_y/df_j = (v_jy - u_y)/rho */
            double A = 0.0, Bx = 0.0, By = 0.0, g = 0.0;
            for (int i = 0; i < Q; ++i) {
                A += L[i] * dr[i];
                Bx += L[i] * dx[i];
                By += L[i] * dy[i];
                g += L[i] * (fs[i] - feq[i]);
            }
            double psi = c, dpsi_db = -2.0, dpsi[9] = {0.0};
            if (a[s] == AUX_FSTAR) {
                psi = 0.0;
                dpsi_db = 0.0;
            } else if (a[s] <= AUX_POS0) {
                /* psi = f*_k / (f*_k - f_k): independent of beta */
                int k = (int)(AUX_POS0 - a[s]);
                double D = feq[k] - fs[k];
                psi = feq[k] / D;
                dpsi_db = 0.0;
                for (int j = 0; j < Q; ++j) {
                    dfk[j] = dr[k] + dx[k] * (cx[j] - ux) / r + dy[k] * (cy[j] - uy) / r;
                    dpsi[j] = (-fs[k] * dfk[j] + (j == k ? feq[k] : 0.0)) / (D * D);
                }
            } else if (a[s] >= 0) {
                /* psi = c sqrt(M / C), C = Delta S here, M = Delta S at m */
                double gradC[9], gradM[9], fm[9];
                double C = delta_s_grad(cfg, fs, gradC);
                gather(Q, f, N, a[s], fm);
                double M = delta_s_grad(cfg, fm, gradM);
                double phi = isinf(C) ? 0.0 : sqrt(M / C);
                psi = c * phi;
                dpsi_db = -2.0 * phi;
                if (!isinf(C) && M > 0.0) {
                    for (int j = 0; j < Q; ++j) dpsi[j] = -c * phi / (2.0 * C) * gradC[j];
                }
            }
            for (int j = 0; j < Q; ++j) {
                double aj = A + Bx * (cx[j] - ux) / r + By * (cy[j] - uy) / r;
                lam[j * N + s] = (1.0 - psi) * aj + psi * L[j] + g * dpsi[j];
            }
            gB += g * dpsi_db;
        }
        /* median: psi of a selected site s depends on f at its median site m
         * through M = Delta S(m): dpsi/df(m)_j = c phi / (2 M) dM/df(m)_j */
        if (cfg->collision == ORC_MEDIAN) {
            for (long long s = 0; s < N; ++s) {
                if (a[s] < 0) continue;
                double fs[9], feq[9], L[9], fm[9], gradM[9];
                gather(Q, f, N, s, fs);
                gather(Q, Lam, N, s, L);
                site_equilibrium(cfg, fs, feq);
                double g = 0.0;
                for (int i = 0; i < Q; ++i) g += L[i] * (fs[i] - feq[i]);
                double C = orc_delta_s(Q, fs, feq);
                gather(Q, f, N, a[s], fm);
                double M = delta_s_grad(cfg, fm, gradM);
                if (isinf(C) || !(M > 0.0)) continue;
                double phi = sqrt(M / C);
                for (int j = 0; j < Q; ++j) lam[j * N + a[s]] += g * c * phi / (2.0 * M) * gradM[j];
            }
        }
    }
    memcpy(dJ_df0, lam, sizeof(double) * S);
    *dJ_dU = gU;
    *dJ_dbeta = gB;
    free(tape); free(aux); free(mask); free(F); free(dS); free(lam); free(Lam);
    return 0;
}
