/*
 * lbm_oracle.c -- plain, slow, FP64 CPU oracle for the Ehrenfest-regularised
 * lattice Boltzmann step (Brownlee, Gorban, Levesley, "Stable simulation of
 * fluid flow with high-Reynolds number using Ehrenfests' steps", 2007).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA path: every lattice table below is typed in here from the paper.
 *
 * Arithmetic is IEEE double (built with -ffp-contract=off so that no fused
 * multiply-add changes the rounding on any host).  Every function follows one
 * passage of the paper, cited in its comment; where the paper is silent or
 * garbled the reading taken is stated at the point of use.
 *
 * One time step, in the paper's textbook order (Sec. 3.2 "Decoupling time
 * step and viscosity", Sec. 4.1 update (lbgkLB) and (ESLB)):
 *   state f(x,t) is PRE-collision;
 *   1. at every fluid site: moments M = m(f), quasiequilibrium f*_M,
 *      nonequilibrium entropy dS = sum_i f_i ln(f_i / f*_i)      (DelS);
 *   2. select the k sites with the largest dS > delta (all of them if
 *      fewer than k qualify)                                         (Sec. 3.2);
 *   3. collide: selected sites jump to f* (Ehrenfests' step), all others
 *      take the LBGK step f + 2 beta (f* - f)                        (ESLB);
 *   4. free flight: f(x, t+1) = f'(x - v_i, t) with the boundary rules of
 *      Sec. 4.2 (exact shift on the grid, Sec. 3.2 last paragraph).
 * With a storage type other than FP64 (the precision form), the
 * post-collision populations of step 3 are rounded to that type before the
 * free flight, as a field stored in that type holds them.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Lattices (Sec. 4.1 for D1Q3, Sec. 4.2 for D2Q9).                    */
/* ------------------------------------------------------------------ */

enum { ORA_D1Q3 = 0, ORA_D2Q9 = 1 };
enum { ORA_EQ_POLY = 0, ORA_EQ_ENTROPIC = 1, ORA_EQ_ENERGY = 2 };
enum { ORA_BC_BB = 0, ORA_BC_FREESLIP = 1, ORA_BC_INLET = 2,
       ORA_BC_OUTLET = 3, ORA_BC_PERIODIC = 4, ORA_BC_OUTLET_COPY = 5 };
enum { ORA_WALL_BOUNCE_BACK = 0, ORA_WALL_DIFFUSE = 1 };

/* D1Q3, paper numbering {v1, v2, v3} = {0, -1, +1} (Sec. 4.1): static,
 * left-moving, right-moving.  The weights are not printed; they are read
 * off the rest-state quasiequilibrium f*(u=0) = rho (2/3, 1/6, 1/6) of the
 * polynomial formulas and the weights inside H of Sec. 4.1. */
static const int    d1_cx[3] = {0, -1, 1};
static const double d1_w[3]  = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0};

/* D2Q9, paper numbering (Sec. 4.2): 0 rest, 1..4 = E, N, W, S (unit
 * speed), 5..8 = NE, NW, SW, SE (speed sqrt 2); weights 4/9, 1/9, 1/36. */
static const int    d2_cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int    d2_cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double d2_w[9]  = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                                1.0 / 9.0, 1.0 / 36.0, 1.0 / 36.0,
                                1.0 / 36.0, 1.0 / 36.0};

int ora_q(int lattice) { return lattice == ORA_D1Q3 ? 3 : 9; }

static int lat_cx(int lattice, int i) { return lattice == ORA_D1Q3 ? d1_cx[i] : d2_cx[i]; }
static int lat_cy(int lattice, int i) { return lattice == ORA_D1Q3 ? 0 : d2_cy[i]; }
static double lat_w(int lattice, int i) { return lattice == ORA_D1Q3 ? d1_w[i] : d2_w[i]; }

/* Index of the population with velocity (cx, cy); -1 if none. */
static int lat_find(int lattice, int cx, int cy)
{
    int q = ora_q(lattice);
    for (int i = 0; i < q; i++)
        if (lat_cx(lattice, i) == cx && lat_cy(lattice, i) == cy) return i;
    return -1;
}

/* Exposed for the tests that pin the tables (sum W = 1, sum W v = 0,
 * sum W v v = 1/3 I). */
void ora_lattice(int lattice, int* cx, int* cy, double* w)
{
    int q = ora_q(lattice);
    for (int i = 0; i < q; i++) {
        cx[i] = lat_cx(lattice, i);
        cy[i] = lat_cy(lattice, i);
        w[i] = lat_w(lattice, i);
    }
}

/* ------------------------------------------------------------------ */
/* Moments (Sec. 2, M = (rho, rho u1, rho u2, 2E); discrete sums of     */
/* Sec. 4.1 and Sec. 4.2).  2E = sum_i |v_i|^2 f_i on the lattice.      */
/* ------------------------------------------------------------------ */
void ora_moments(int lattice, const double* f, double* M)
{
    int q = ora_q(lattice);
    double rho = 0, jx = 0, jy = 0, e2 = 0;
    for (int i = 0; i < q; i++) {
        double cx = lat_cx(lattice, i), cy = lat_cy(lattice, i);
        rho += f[i];
        jx += cx * f[i];
        jy += cy * f[i];
        e2 += (cx * cx + cy * cy) * f[i];
    }
    M[0] = rho; M[1] = jx; M[2] = jy; M[3] = e2;
}

/* ------------------------------------------------------------------ */
/* Quasiequilibria.                                                     */
/* ------------------------------------------------------------------ */

/* Polynomial quasiequilibrium.  D1Q3: the three formulas of Sec. 4.1.
 * D2Q9: not printed in the paper (it cites the textbook of Succi); the
 * standard second-order form W_i rho (1 + 3 v.u + 9/2 (v.u)^2 - 3/2 u^2)
 * is used, whose 1-D restriction is exactly the D1Q3 formulas. */
static void feq_poly(int lattice, double rho, double ux, double uy, double* fs)
{
    if (lattice == ORA_D1Q3) {
        fs[0] = 2.0 * rho / 3.0 * (1.0 - 1.5 * ux * ux);
        fs[1] = rho / 6.0 * (1.0 - 3.0 * ux + 3.0 * ux * ux);
        fs[2] = rho / 6.0 * (1.0 + 3.0 * ux + 3.0 * ux * ux);
        return;
    }
    double usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; i++) {
        double cu = d2_cx[i] * ux + d2_cy[i] * uy;
        fs[i] = d2_w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

/* Entropic quasiequilibrium for mass and momentum.
 * D1Q3: the explicit maximiser of S = -H, H = f1 log(f1/4) + f2 log f2 +
 * f3 log f3 (Sec. 4.1).  As printed, the formulas for f2* and f3* carry
 * swapped labels (their difference is -rho u); the reading used here puts
 * them on the populations whose momentum is +rho u:
 *   rest  f1* = (2 rho / 3)(2 - s),
 *   left  f2* = (rho / 6)(2 s - 3 u - 1),
 *   right f3* = (rho / 6)(3 u - 1 + 2 s),      s = sqrt(1 + 3 u^2).
 * D2Q9: the product formula of Sec. 4.2,
 *   f*_i = rho W_i prod_j (2 - s_j) ((2 u_j + s_j) / (1 - u_j))^{v_ij}. */
static void feq_entropic(int lattice, double rho, double ux, double uy, double* fs)
{
    if (lattice == ORA_D1Q3) {
        double s = sqrt(1.0 + 3.0 * ux * ux);
        fs[0] = 2.0 * rho / 3.0 * (2.0 - s);
        fs[1] = rho / 6.0 * (2.0 * s - 3.0 * ux - 1.0);
        fs[2] = rho / 6.0 * (3.0 * ux - 1.0 + 2.0 * s);
        return;
    }
    double u[2] = {ux, uy};
    double a[2], b[2];
    for (int j = 0; j < 2; j++) {
        double s = sqrt(1.0 + 3.0 * u[j] * u[j]);
        a[j] = 2.0 - s;
        b[j] = (2.0 * u[j] + s) / (1.0 - u[j]);
    }
    for (int i = 0; i < 9; i++) {
        int v[2] = {d2_cx[i], d2_cy[i]};
        double p = rho * d2_w[i];
        for (int j = 0; j < 2; j++) {
            p *= a[j];
            if (v[j] == 1) p *= b[j];
            else if (v[j] == -1) p /= b[j];
        }
        fs[i] = p;
    }
}

/* Entropic quasiequilibrium with the energy constraint: the maximiser of
 * the perfect entropy S = -sum f ln(f/W) (PerfEnt) subject to m(f) = M with
 * M = (rho, rho u1, rho u2, 2E) (argmax).  Its Lagrange form (Sec. 3.3) is
 * ln(f*_i / W_i) = sum_j mu_j m_j(v_i), m(v) = (1, v_x, v_y, |v|^2) (the
 * printed form drops W_i; it is restored here so that mu = 0 is the rest
 * state of unit density).  mu is the unique minimiser of the strictly
 * convex dual  Phi(mu) = sum_i W_i exp(mu . m_i) - mu . M;  Newton's method
 * with a backtracking line search on Phi is used.  For D1Q3 the moment
 * vector is (rho, rho u, 2E) and mu has three entries; D2Q9 uses four.
 *   mu  : in = start point, out = solution.
 *   returns iterations used, or -1 when the residual did not reach tol
 *   (max-norm of m(f*) - M divided by rho) within maxit iterations. */
static int nmom(int lattice) { return lattice == ORA_D1Q3 ? 3 : 4; }

static void energy_feq_from_mu(int lattice, const double* mu, double* fs)
{
    int q = ora_q(lattice);
    for (int i = 0; i < q; i++) {
        double cx = lat_cx(lattice, i), cy = lat_cy(lattice, i);
        double arg;
        if (lattice == ORA_D1Q3)
            arg = mu[0] + mu[1] * cx + mu[2] * cx * cx;
        else
            arg = mu[0] + mu[1] * cx + mu[2] * cy + mu[3] * (cx * cx + cy * cy);
        fs[i] = lat_w(lattice, i) * exp(arg);
    }
}

static void moment_vector(int lattice, int i, double* m)
{
    double cx = lat_cx(lattice, i), cy = lat_cy(lattice, i);
    if (lattice == ORA_D1Q3) {
        m[0] = 1.0; m[1] = cx; m[2] = cx * cx;
    } else {
        m[0] = 1.0; m[1] = cx; m[2] = cy; m[3] = cx * cx + cy * cy;
    }
}

static double dual_phi(int lattice, const double* mu, const double* Mv)
{
    int q = ora_q(lattice), nm = nmom(lattice);
    double fs[9], phi = 0.0;
    energy_feq_from_mu(lattice, mu, fs);
    for (int i = 0; i < q; i++) phi += fs[i];
    for (int j = 0; j < nm; j++) phi -= mu[j] * Mv[j];
    return phi;
}

/* Solve the small symmetric positive definite system J x = r by Cholesky
 * factorisation (textbook; n <= 4). Returns 0, or -1 if J is not SPD. */
static int spd_solve(int n, const double* J, const double* r, double* x)
{
    double L[16] = {0};
    for (int i = 0; i < n; i++) {
        for (int j = 0; j <= i; j++) {
            double s = J[i * n + j];
            for (int k = 0; k < j; k++) s -= L[i * 4 + k] * L[j * 4 + k];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                L[i * 4 + i] = sqrt(s);
            } else {
                L[i * 4 + j] = s / L[j * 4 + j];
            }
        }
    }
    double y[4];
    for (int i = 0; i < n; i++) {
        double s = r[i];
        for (int k = 0; k < i; k++) s -= L[i * 4 + k] * y[k];
        y[i] = s / L[i * 4 + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = y[i];
        for (int k = i + 1; k < n; k++) s -= L[k * 4 + i] * x[k];
        x[i] = s / L[i * 4 + i];
    }
    return 0;
}

/* Max-norm residual of the moment constraints divided by rho. */
static double newton_residual(int lattice, const double* mu, const double* Mv, double* r)
{
    int q = ora_q(lattice), nm = nmom(lattice);
    double fs[9];
    energy_feq_from_mu(lattice, mu, fs);
    for (int j = 0; j < nm; j++) r[j] = -Mv[j];
    for (int i = 0; i < q; i++) {
        double m[4];
        moment_vector(lattice, i, m);
        for (int j = 0; j < nm; j++) r[j] += m[j] * fs[i];
    }
    double rn = 0.0;
    for (int j = 0; j < nm; j++) rn = fmax(rn, fabs(r[j]));
    return rn / Mv[0];
}

int ora_newton(int lattice, const double* Mv, double* mu, double tol, int maxit)
{
    int q = ora_q(lattice), nm = nmom(lattice);
    double r[4];
    for (int it = 0; it <= maxit; it++) {
        double rn = newton_residual(lattice, mu, Mv, r);
        if (rn <= tol) return it;
        if (it == maxit) break;
        double fs[9], J[16] = {0}, step[4];
        energy_feq_from_mu(lattice, mu, fs);
        for (int i = 0; i < q; i++) {
            double m[4];
            moment_vector(lattice, i, m);
            for (int a = 0; a < nm; a++)
                for (int b = 0; b < nm; b++) J[a * nm + b] += m[a] * m[b] * fs[i];
        }
        if (spd_solve(nm, J, r, step) != 0) return -1;
        /* Backtracking on the dual objective (Armijo).  Near the root the
         * decrease of Phi falls below its rounding, so a step that shrinks
         * the residual is accepted as well. */
        double phi0 = dual_phi(lattice, mu, Mv);
        double slope = 0.0;
        for (int j = 0; j < nm; j++) slope += r[j] * step[j];
        double t = 1.0, trial[4], rt[4];
        for (int ls = 0; ls < 60; ls++) {
            for (int j = 0; j < nm; j++) trial[j] = mu[j] - t * step[j];
            if (dual_phi(lattice, trial, Mv) <= phi0 - 1e-4 * t * slope) break;
            if (newton_residual(lattice, trial, Mv, rt) < rn) break;
            t *= 0.5;
        }
        for (int j = 0; j < nm; j++) mu[j] = trial[j];
    }
    return -1;
}

/* Polynomial start point for Newton (the paper does not define one): the
 * multipliers of the first-order expansion of the quasiequilibrium about
 * rest, mu0 = (ln rho - 3/2 u^2, 3 u_x, 3 u_y, 0) (D1Q3: (ln rho - 3/2 u^2,
 * 3u, 0)). */
void ora_mu_guess(int lattice, const double* Mv, double* mu)
{
    double rho = Mv[0];
    if (lattice == ORA_D1Q3) {
        double u = Mv[1] / rho;
        mu[0] = log(rho) - 1.5 * u * u; mu[1] = 3.0 * u; mu[2] = 0.0;
    } else {
        double ux = Mv[1] / rho, uy = Mv[2] / rho;
        mu[0] = log(rho) - 1.5 * (ux * ux + uy * uy);
        mu[1] = 3.0 * ux; mu[2] = 3.0 * uy; mu[3] = 0.0;
    }
}

#define ORA_NEWTON_TOL 1e-12
#define ORA_NEWTON_MAXIT 100

/* Quasiequilibrium for the moments M (rho, rho ux, rho uy, 2E).
 * eq = POLY / ENTROPIC use rho and u only; ENERGY also matches 2E.
 * Returns 0, or -1 if the energy Newton solve failed. */
int ora_equilibrium(int lattice, int eq, const double* Mv, double* fs)
{
    double rho = Mv[0];
    double ux = Mv[1] / rho;
    double uy = lattice == ORA_D1Q3 ? 0.0 : Mv[2] / rho;
    if (eq == ORA_EQ_POLY) { feq_poly(lattice, rho, ux, uy, fs); return 0; }
    if (eq == ORA_EQ_ENTROPIC) { feq_entropic(lattice, rho, ux, uy, fs); return 0; }
    double Mn[4], mu[4];
    if (lattice == ORA_D1Q3) { Mn[0] = Mv[0]; Mn[1] = Mv[1]; Mn[2] = Mv[3]; }
    else { Mn[0] = Mv[0]; Mn[1] = Mv[1]; Mn[2] = Mv[2]; Mn[3] = Mv[3]; }
    ora_mu_guess(lattice, Mn, mu);
    if (ora_newton(lattice, Mn, mu, ORA_NEWTON_TOL, ORA_NEWTON_MAXIT) < 0) return -1;
    /* polish: up to two more Newton steps toward the rounding floor (the
     * multipliers are then accurate to ~1e-15, well inside the 1e-12 target) */
    ora_newton(lattice, Mn, mu, 1e-15, 2);
    energy_feq_from_mu(lattice, mu, fs);
    return 0;
}

/* Equilibrium from (rho, u) for boundary data: POLY and ENTROPIC use their
 * formulas; the energy form uses the isothermal entropic formula (its 2E
 * is the isothermal energy, where the energy multiplier vanishes). */
static void feq_rho_u(int lattice, int eq, double rho, double ux, double uy, double* fs)
{
    if (eq == ORA_EQ_POLY) feq_poly(lattice, rho, ux, uy, fs);
    else feq_entropic(lattice, rho, ux, uy, fs);
}

void ora_feq_rho_u(int lattice, int eq, double rho, double ux, double uy, double* fs)
{
    feq_rho_u(lattice, eq, rho, ux, uy, fs);
}

/* ------------------------------------------------------------------ */
/* Entropies.                                                           */
/* ------------------------------------------------------------------ */

/* Perfect entropy S(f) = -sum_i f_i ln(f_i / W_i) (PerfEnt), with
 * 0 ln 0 = 0.  Returns -inf when some f_i < 0 (outside the domain). */
double ora_perfect_entropy(int lattice, const double* f)
{
    int q = ora_q(lattice);
    double s = 0.0;
    for (int i = 0; i < q; i++) {
        if (f[i] < 0.0) return -INFINITY;
        if (f[i] > 0.0) s -= f[i] * log(f[i] / lat_w(lattice, i));
    }
    return s;
}

/* Nonequilibrium entropy dS = sum_i f_i ln(f_i / f*_i) (DelS, the minus
 * Kullback entropy; Sec. 3.3 uses it for entropic and non-entropic f*).
 * The paper does not treat states outside the positive cone (polynomial
 * LBGK near beta = 1 can produce them): such a site is read as maximally
 * far from equilibrium, dS = +inf, when some f_i < 0 or some f*_i <= 0.
 * A zero population contributes 0 (0 ln 0 = 0). */
double ora_delta_s(int lattice, const double* f, const double* fs)
{
    int q = ora_q(lattice);
    for (int i = 0; i < q; i++)
        if (f[i] < 0.0 || !(fs[i] > 0.0)) return INFINITY;
    double s = 0.0;
    for (int i = 0; i < q; i++)
        if (f[i] > 0.0) s += f[i] * log(f[i] / fs[i]);
    return s;
}

/* ------------------------------------------------------------------ */
/* Selection of the Ehrenfests' sites (Sec. 3.2 last paragraph, Sec.   */
/* 4.1 below (ESLB)): among eligible sites with dS > delta (strict),   */
/* the k with the largest dS; all of them if fewer than k qualify.     */
/* The paper is silent on ties: the total order (dS descending, site   */
/* index ascending) is used.  Output indices are sorted ascending.     */
/* ------------------------------------------------------------------ */
/* ELBM (elbmLB): the parameter alpha of f + alpha beta (f* - f) solves the
 * constant-entropy condition S(f + alpha (f* - f)) = S(f) (nontrivial root).
 * With D = f* - f, x_i = alpha D_i / f_i and phi(x) = (1+x) ln(1+x) - x, and
 * sum D = 0 (f* has the moments of f), the condition reads
 *     sum f_i phi(alpha D_i / f_i) = alpha sum D_i ln(1 + D_i / f_i)
 * (the left side minus the right side is -(S(f + alpha D) - S(f)), with
 * no cancellation between two entropies).  Its left side over alpha is
 * increasing (phi is convex, phi(0) = 0), so the root above alpha = 1 is
 * unique.  Bisection (the paper's method) on [1, alpha_max] to 1e-15, with
 * alpha_max the largest alpha keeping f + alpha D >= 0; when the entropy
 * still exceeds S(f) at alpha_max, alpha = alpha_max.  f = f* (D = 0) gives
 * the LBGK value alpha = 2.  Returns alpha; -1 for f outside the positive
 * cone (f_i <= 0). */
/* phi(x) = (1 + x) ln(1 + x) - x for x >= -1 (phi(-1) = 1); for |x| < 0.05
 * its Taylor series sum_{n>=2} (-1)^n x^n / (n (n-1)) to n = 16 (the
 * direct form loses the leading x^2 / 2 to cancellation there). */
static double phi(double x)
{
    if (x <= -1.0) return 1.0;
    if (fabs(x) < 0.05) {
        double s = 0.0, p = x * x;
        for (int n = 2; n <= 16; n++) {
            s += ((n & 1) ? -1.0 : 1.0) * p / (double)(n * (n - 1));
            p *= x;
        }
        return s;
    }
    return (1.0 + x) * log1p(x) - x;
}

static double elbm_gap(int q, const double* f, const double* D, double R, double alpha)
{
    double s = 0.0;
    for (int i = 0; i < q; i++) s += f[i] * phi(alpha * D[i] / f[i]);
    return s - alpha * R;
}

double ora_elbm_alpha(int lattice, const double* f, const double* fs)
{
    int q = ora_q(lattice);
    double D[9], R = 0.0, amax = INFINITY;
    int moved = 0;
    for (int i = 0; i < q; i++) {
        if (!(f[i] > 0.0) || !(fs[i] > 0.0)) return -1.0;
        D[i] = fs[i] - f[i];
        if (D[i] != 0.0) moved = 1;
        if (D[i] < 0.0) amax = fmin(amax, f[i] / -D[i]);
        R += D[i] * log1p(D[i] / f[i]);
    }
    if (!moved || !(R > 0.0)) return 2.0;
    double lo = 1.0, hi = amax;
    if (!isfinite(hi)) return 2.0;
    if (elbm_gap(q, f, D, R, hi) <= 0.0) return hi;    /* no root before the positivity limit */
    while (hi - lo > 1e-15 * hi) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (elbm_gap(q, f, D, R, mid) <= 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

typedef struct { double ds; long idx; } cand_t;

static int cand_cmp(const void* pa, const void* pb)
{
    const cand_t* a = (const cand_t*)pa;
    const cand_t* b = (const cand_t*)pb;
    if (a->ds > b->ds) return -1;
    if (a->ds < b->ds) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

static int long_cmp(const void* pa, const void* pb)
{
    long a = *(const long*)pa, b = *(const long*)pb;
    return (a > b) - (a < b);
}

long ora_select(const double* ds, const unsigned char* eligible, long n,
                double delta, long k, long* idx_out)
{
    if (k <= 0) return 0;
    cand_t* c = (cand_t*)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
    long nc = 0;
    for (long i = 0; i < n; i++) {
        if (eligible && !eligible[i]) continue;
        if (ds[i] > delta) { c[nc].ds = ds[i]; c[nc].idx = i; nc++; }
    }
    qsort(c, (size_t)nc, sizeof(cand_t), cand_cmp);
    long m = nc < k ? nc : k;
    for (long i = 0; i < m; i++) idx_out[i] = c[i].idx;
    free(c);
    qsort(idx_out, (size_t)m, sizeof(long), long_cmp);
    return m;
}

/* ------------------------------------------------------------------ */
/* Run configuration and the time step.                                 */
/* ------------------------------------------------------------------ */
typedef struct {
    int lattice;     /* ORA_D1Q3 / ORA_D2Q9 */
    int nx, ny;      /* ny = 1 for D1Q3 */
    int eq;          /* ORA_EQ_* */
    double beta;     /* LBGK parameter of (lbgkLB) */
    double delta;    /* Ehrenfests' tolerance */
    long k;          /* sites per step */
    int bc[4];       /* x = 0, x = nx-1, y = 0, y = ny-1 */
    double rho_in, ux_in, uy_in;   /* inlet state */
    int ox0, oy0, ow, oh;          /* solid rectangle; ow == 0: none */
    int elbm;                      /* collision (elbmLB) instead of (lbgkLB) */
    int wall;                      /* rule on the rectangle's faces: ORA_WALL_* */
    int store;                     /* storage of the populations: ORA_STORE_* */
} ora_cfg;

/* ------------------------------------------------------------------ */
/* Storage of the populations (the precision form: populations stored  */
/* in FP32 or FP16, as f or as deviations f - W_i rho0 with rho0 = 1).  */
/* The method computes in exact (here FP64) arithmetic; what a stored   */
/* field can hold is the value rounded to the storage type, once per    */
/* time step, when the post-collision populations are written.          */
/* ------------------------------------------------------------------ */
enum { ORA_STORE_F64 = 0, ORA_STORE_F32 = 1, ORA_STORE_F32_DEV = 2, ORA_STORE_F16_DEV = 3 };

/* Round to nearest, ties to even, to a binary floating-point format with
 * p significand bits and smallest normal exponent emin (IEEE 754 binary32:
 * p = 24, emin = -126; binary16: p = 11, emin = -14), overflow to +-inf at
 * max_finite.  Written from the format's definition: below 2^emin the
 * spacing is the subnormal quantum 2^(emin - p + 1); above it, the spacing
 * is 2^(e - p + 1) for x in [2^e, 2^(e+1)).  nearbyint rounds ties to even
 * in the default rounding mode. */
static double round_to_format(double x, int p, int emin, double max_finite)
{
    if (!isfinite(x) || x == 0.0) return x;
    int e;
    frexp(x, &e);             /* |x| in [2^(e-1), 2^e) */
    e -= 1;
    if (e < emin) e = emin;
    double q = ldexp(1.0, e - p + 1);
    double r = nearbyint(x / q) * q;   /* x / q and r * q are exact scalings */
    if (fabs(r) > max_finite) {
        /* beyond the largest finite value: rounds to infinity at and above
         * max_finite + half its spacing */
        double half = ldexp(1.0, (int)(log2(max_finite)) - p);
        if (fabs(x) >= max_finite + half) return x > 0 ? INFINITY : -INFINITY;
        return x > 0 ? max_finite : -max_finite;
    }
    return r;
}

double ora_round_f32(double x) { return round_to_format(x, 24, -126, 3.4028234663852886e38); }
double ora_round_f16(double x) { return round_to_format(x, 11, -14, 65504.0); }

/* Value of one stored population of weight w (rho0 = 1 for the deviation
 * forms). */
static double stored_value(int store, double f, double w)
{
    switch (store) {
        case ORA_STORE_F32: return ora_round_f32(f);
        case ORA_STORE_F32_DEV: return w + ora_round_f32(f - w);
        case ORA_STORE_F16_DEV: return w + ora_round_f16(f - w);
        default: return f;
    }
}

static int is_solid(const ora_cfg* c, int x, int y)
{
    return c->ow > 0 && x >= c->ox0 && x < c->ox0 + c->ow &&
           y >= c->oy0 && y < c->oy0 + c->oh;
}

static long site(const ora_cfg* c, int x, int y) { return (long)y * c->nx + x; }

/* Pre-collision populations at fluid site (x, y) at time t+1 from the
 * post-collision field fp at time t: free flight f_i(x) = fp_i(x - v_i)
 * (Sec. 3, Theta_tau; exact on the grid, Sec. 3.2) with these rules where
 * x - v_i leaves the fluid (Sec. 4.2, boundary paragraph):
 *  - x side INLET : incoming populations take the quasiequilibrium of the
 *                   free stream (rho_in, u_in);
 *  - x side OUTLET: incoming populations take the quasiequilibrium of the
 *                   density and velocity of the penultimate column (x = nx-2,
 *                   same row) of the post-collision field;
 *  - x side OUTLET_COPY (zero-gradient outflow; the paper's outlet is the
 *                   one above): the column beyond the side is read as a copy
 *                   of the side column (source column x instead of x - v_x),
 *                   then the y and obstacle rules apply as usual;
 *  - BB           : half-way bounce-back, f_i(x) = fp_{-i}(x);
 *  - PERIODIC     : wrap around;
 *  - y side FREESLIP: specular reflection, the population (v_x, -v_y) that
 *                   left (x - v_x, y) arrives as (v_x, v_y);
 *  - solid source : half-way bounce-back (the paper leaves the cylinder
 *                   wall rule open; no-slip bounce-back is the reading),
 *                   or, with wall = ORA_WALL_DIFFUSE, the diffuse kinetic
 *                   wall of the references of Sec. 4.2 (below).
 * The x rule is applied first (inlet/outlet take precedence at corners).
 *
 * Diffuse wall (Maxwell's diffuse reflection on a wall at rest): the
 * populations that enter x from the wall are the wall's quasiequilibrium at
 * rest, f_i(x) = W_i rho_w (every quasiequilibrium of this library is
 * W_i rho at u = 0), and rho_w makes the wall impermeable: what enters
 * equals what the wall absorbed, the post-collision populations f'_{-i}(x)
 * of the same links, so
 *     f_i(x) = W_i (sum_{j in B} f'_{-j}(x)) / (sum_{j in B} W_j),
 * B the directions i whose source x - v_i is solid.  On a face every such
 * link has |v . n| = 1, so the flux weights of the kinetic rule are all one;
 * at a convex corner B is the one diagonal link (the same rule). */
static void gather_site(const ora_cfg* c, const double* fp, int x, int y, double* f)
{
    int L = c->lattice, q = ora_q(L), nx = c->nx, ny = c->ny;
    long N = (long)nx * ny, s0 = site(c, x, y);
    int wall_link[9] = {0};
    int nwall = 0;
    for (int i = 0; i < q; i++) {
        int cx = lat_cx(L, i), cy = lat_cy(L, i);
        int sx = x - cx, sy = y - cy;
        if (sx < 0 || sx >= nx) {
            int kind = sx < 0 ? c->bc[0] : c->bc[1];
            if (kind == ORA_BC_PERIODIC) {
                sx = (sx + nx) % nx;
            } else if (kind == ORA_BC_INLET) {
                double fs[9];
                feq_rho_u(L, c->eq, c->rho_in, c->ux_in, c->uy_in, fs);
                f[i] = fs[i];
                continue;
            } else if (kind == ORA_BC_OUTLET) {
                double g[9], M[4], fs[9];
                long sp = site(c, nx - 2, y);
                for (int j = 0; j < q; j++) g[j] = fp[j * N + sp];
                ora_moments(L, g, M);
                feq_rho_u(L, c->eq, M[0], M[1] / M[0], L == ORA_D1Q3 ? 0.0 : M[2] / M[0], fs);
                f[i] = fs[i];
                continue;
            } else if (kind == ORA_BC_OUTLET_COPY) {
                sx = x;
            } else { /* BB (FREESLIP is not accepted on x sides) */
                int o = lat_find(L, -cx, -cy);
                f[i] = fp[o * N + s0];
                continue;
            }
        }
        if (sy < 0 || sy >= ny) {
            int kind = sy < 0 ? c->bc[2] : c->bc[3];
            if (kind == ORA_BC_PERIODIC) {
                sy = (sy + ny) % ny;
            } else if (kind == ORA_BC_FREESLIP) {
                int m = lat_find(L, cx, -cy);
                f[i] = fp[m * N + site(c, sx, y)];
                continue;
            } else { /* BB */
                int o = lat_find(L, -cx, -cy);
                f[i] = fp[o * N + s0];
                continue;
            }
        }
        if (is_solid(c, sx, sy)) {
            int o = lat_find(L, -cx, -cy);
            f[i] = fp[o * N + s0];
            if (c->wall == ORA_WALL_DIFFUSE) { wall_link[i] = 1; nwall++; }
            continue;
        }
        f[i] = fp[i * N + site(c, sx, sy)];
    }
    if (nwall > 0) {
        /* f[i] holds f'_{-i}(x) on the wall links (read above) */
        double absorbed = 0.0, wsum = 0.0;
        for (int i = 0; i < q; i++)
            if (wall_link[i]) { absorbed += f[i]; wsum += lat_w(L, i); }
        double rho_w = absorbed / wsum;
        for (int i = 0; i < q; i++)
            if (wall_link[i]) f[i] = lat_w(L, i) * rho_w;
    }
}

/* Field-level helpers exposed to the tests. */

/* Quasiequilibrium and dS at every fluid site of a pre-collision field.
 * Solid sites get fs = 0 and dS = NaN.  Returns the number of sites where
 * the energy Newton solve failed. */
long ora_fields(const ora_cfg* c, const double* f, double* fs_out, double* ds_out)
{
    int L = c->lattice, q = ora_q(L);
    long N = (long)c->nx * c->ny, fails = 0;
#pragma omp parallel for schedule(static) reduction(+:fails)
    for (long s = 0; s < N; s++) {
        int x = (int)(s % c->nx), y = (int)(s / c->nx);
        if (is_solid(c, x, y)) {
            for (int i = 0; i < q; i++) if (fs_out) fs_out[i * N + s] = 0.0;
            if (ds_out) ds_out[s] = NAN;
            continue;
        }
        double g[9], M[4], fs[9];
        for (int i = 0; i < q; i++) g[i] = f[i * N + s];
        ora_moments(L, g, M);
        if (ora_equilibrium(L, c->eq, M, fs) != 0) fails++;
        if (fs_out) for (int i = 0; i < q; i++) fs_out[i * N + s] = fs[i];
        if (ds_out) ds_out[s] = ora_delta_s(L, g, fs);
    }
    return fails;
}

/* Moments of a pre-collision field; solid sites get zeros. */
void ora_moment_fields(const ora_cfg* c, const double* f, double* rho, double* ux,
                       double* uy, double* e2)
{
    int L = c->lattice, q = ora_q(L);
    long N = (long)c->nx * c->ny;
    for (long s = 0; s < N; s++) {
        int x = (int)(s % c->nx), y = (int)(s / c->nx);
        double g[9], M[4] = {0, 0, 0, 0};
        if (!is_solid(c, x, y)) {
            for (int i = 0; i < q; i++) g[i] = f[i * N + s];
            ora_moments(L, g, M);
        }
        rho[s] = M[0];
        ux[s] = M[0] != 0.0 ? M[1] / M[0] : 0.0;
        if (uy) uy[s] = M[0] != 0.0 ? M[2] / M[0] : 0.0;
        if (e2) e2[s] = M[3];
    }
}

/* Initial state: the quasiequilibrium of (rho, ux, uy) at every fluid
 * site (the shock tube and the cylinder both start on the manifold,
 * Sec. 4.1 and Sec. 4.2).  e2 (nullable) gives 2E for the energy form;
 * when NULL the isothermal energy of the entropic formula is used. */
int ora_init(const ora_cfg* c, const double* rho, const double* ux, const double* uy,
             const double* e2, double* f)
{
    int L = c->lattice, q = ora_q(L);
    long N = (long)c->nx * c->ny;
    int bad = 0;
    for (long s = 0; s < N; s++) {
        int x = (int)(s % c->nx), y = (int)(s / c->nx);
        double fs[9];
        if (is_solid(c, x, y)) {
            for (int i = 0; i < q; i++) f[i * N + s] = 0.0;
            continue;
        }
        double vy = (L == ORA_D1Q3 || !uy) ? 0.0 : uy[s];
        if (c->eq == ORA_EQ_ENERGY && e2) {
            double M[4] = {rho[s], rho[s] * ux[s], rho[s] * vy, e2[s]};
            if (ora_equilibrium(L, c->eq, M, fs) != 0) bad = 1;
        } else {
            feq_rho_u(L, c->eq, rho[s], ux[s], vy, fs);
        }
        for (int i = 0; i < q; i++) f[i * N + s] = fs[i];
    }
    return bad ? -1 : 0;
}

/* Advance the pre-collision field f by nsteps steps (see the file head).
 *   replay_cnt/replay_idx (nullable): when given, step t uses the listed
 *     sites (replay_cnt[t] of them, concatenated) instead of selecting;
 *   cnt_log[t]  (nullable): number of sites that took the Ehrenfests' step;
 *   sel_log     (nullable): their indices, concatenated, ascending per
 *     step, at most sel_cap in total;
 *   probe_log[t] (nullable): u_x of the pre-collision state at (px, py)
 *     at the start of step t.
 * Returns 0, -1 on a Newton failure, -2 on a non-finite population,
 * -3 when sel_log overflows. */
int ora_run(const ora_cfg* c, double* f, long nsteps,
            const long* replay_cnt, const long* replay_idx,
            long* cnt_log, long* sel_log, long sel_cap,
            double* probe_log, int px, int py)
{
    int L = c->lattice, q = ora_q(L), nx = c->nx, ny = c->ny;
    long N = (long)nx * ny;
    double* fs = (double*)malloc(sizeof(double) * (size_t)(q * N));
    double* fp = (double*)malloc(sizeof(double) * (size_t)(q * N));
    double* ds = (double*)malloc(sizeof(double) * (size_t)N);
    unsigned char* elig = (unsigned char*)malloc((size_t)N);
    unsigned char* chosen = (unsigned char*)malloc((size_t)N);
    long* sel = (long*)malloc(sizeof(long) * (size_t)(c->k > 0 ? c->k : 1));
    int status = 0;
    long sel_used = 0, replay_off = 0;
    for (long s = 0; s < N; s++)
        elig[s] = !is_solid(c, (int)(s % nx), (int)(s / nx));

    for (long t = 0; t < nsteps && status == 0; t++) {
        if (probe_log) {
            double g[9], M[4];
            long sp = site(c, px, py);
            for (int i = 0; i < q; i++) g[i] = f[i * N + sp];
            ora_moments(L, g, M);
            probe_log[t] = M[1] / M[0];
        }
        /* 1. moments, quasiequilibrium and dS at every fluid site */
        if (ora_fields(c, f, fs, ds) != 0) { status = -1; break; }
        /* 2. selection */
        long m;
        if (replay_cnt) {
            m = replay_cnt[t];
            for (long j = 0; j < m; j++) sel[j] = replay_idx[replay_off + j];
            replay_off += m;
        } else {
            m = ora_select(ds, elig, N, c->delta, c->k, sel);
        }
        memset(chosen, 0, (size_t)N);
        for (long j = 0; j < m; j++) chosen[sel[j]] = 1;
        if (cnt_log) cnt_log[t] = m;
        if (sel_log) {
            if (sel_used + m > sel_cap) { status = -3; break; }
            for (long j = 0; j < m; j++) sel_log[sel_used + j] = sel[j];
            sel_used += m;
        }
        /* 3. collision: Ehrenfests' step at chosen sites, LBGK (or ELBM)
         *    elsewhere */
#pragma omp parallel for schedule(static)
        for (long s = 0; s < N; s++) {
            double a = 2.0;
            if (c->elbm && elig[s] && !chosen[s]) {
                double gl[9], gs[9];
                for (int i = 0; i < q; i++) { gl[i] = f[i * N + s]; gs[i] = fs[i * N + s]; }
                a = ora_elbm_alpha(L, gl, gs);
                if (a < 0.0) a = 2.0;   /* outside the positive cone: dS = +inf, LBGK */
            }
            for (int i = 0; i < q; i++) {
                double fi = f[i * N + s], fsi = fs[i * N + s];
                if (!elig[s]) fp[i * N + s] = 0.0;
                else if (chosen[s]) fp[i * N + s] = fsi;
                else fp[i * N + s] = fi + a * c->beta * (fsi - fi);
                if (c->store != ORA_STORE_F64 && elig[s])
                    fp[i * N + s] = stored_value(c->store, fp[i * N + s], lat_w(L, i));
            }
        }
        /* 4. free flight with boundary rules */
        int nonfinite = 0;
#pragma omp parallel for schedule(static) reduction(|:nonfinite)
        for (long s = 0; s < N; s++) {
            int x = (int)(s % nx), y = (int)(s / nx);
            double g[9];
            if (!elig[s]) {
                for (int i = 0; i < q; i++) f[i * N + s] = 0.0;
                continue;
            }
            gather_site(c, fp, x, y, g);
            for (int i = 0; i < q; i++) {
                f[i * N + s] = g[i];
                if (!isfinite(g[i])) nonfinite = 1;
            }
        }
        if (nonfinite) status = -2;
    }
    free(fs); free(fp); free(ds); free(elig); free(chosen); free(sel);
    return status;
}

/* One collision (no streaming) of a pre-collision field with the given
 * selection: the post-collision field f' of (ESLB).  Used by the tests
 * that check per-site conservation and the Ehrenfests' step. */
int ora_collide(const ora_cfg* c, const double* f, const long* sel, long m, double* fp)
{
    int L = c->lattice, q = ora_q(L);
    long N = (long)c->nx * c->ny;
    double* fs = (double*)malloc(sizeof(double) * (size_t)(q * N));
    unsigned char* chosen = (unsigned char*)calloc((size_t)N, 1);
    int st = ora_fields(c, f, fs, NULL) == 0 ? 0 : -1;
    for (long j = 0; j < m; j++) chosen[sel[j]] = 1;
    for (long s = 0; s < N; s++) {
        int solid = is_solid(c, (int)(s % c->nx), (int)(s / c->nx));
        for (int i = 0; i < q; i++) {
            double fi = f[i * N + s], fsi = fs[i * N + s];
            if (solid) fp[i * N + s] = 0.0;
            else if (chosen[s]) fp[i * N + s] = fsi;
            else {
                double a = 2.0;
                if (c->elbm) {
                    double gl[9], gs[9];
                    for (int j = 0; j < q; j++) { gl[j] = f[j * N + s]; gs[j] = fs[j * N + s]; }
                    a = ora_elbm_alpha(L, gl, gs);
                    if (a < 0.0) a = 2.0;
                }
                fp[i * N + s] = fi + a * c->beta * (fsi - fi);
            }
        }
    }
    free(fs); free(chosen);
    return st;
}

/* Free flight with boundary rules only: pre-collision field at t+1 from a
 * post-collision field fp at t. */
void ora_stream(const ora_cfg* c, const double* fp, double* f)
{
    int L = c->lattice, q = ora_q(L);
    long N = (long)c->nx * c->ny;
    for (long s = 0; s < N; s++) {
        int x = (int)(s % c->nx), y = (int)(s / c->nx);
        double g[9];
        if (is_solid(c, x, y)) {
            for (int i = 0; i < q; i++) f[i * N + s] = 0.0;
            continue;
        }
        gather_site(c, fp, x, y, g);
        for (int i = 0; i < q; i++) f[i * N + s] = g[i];
    }
}

int ora_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
