/*
 * wb_oracle.c -- plain FP64 CPU oracle of the well-balanced phase-field
 * lattice Boltzmann model for incompressible binary fluids
 * (Ju, Liu, Yan, Bao, Sun, Guo; arXiv:2311.10827, Section 2.3).
 *
 * TEST INFRASTRUCTURE.  This file is the independent checker of the CUDA
 * library.  Only the tests, the package smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or constant
 * generator with the CUDA path, and the CUDA path never calls it.
 *
 * Names follow the paper: f is the Cahn-Hilliard (CH) population (Eq. BGK),
 * g the hydrodynamic population (Eq. BGK-NS).
 *
 * State convention.  f[i*N + n] and g[i*N + n] hold the paper's f_i(x,t) and
 * g_i(x,t): populations at time t after streaming, before collision.  S_prev
 * holds u.grad(phi) of the previous step (see reading R1 below).  Nodes are
 * numbered n = (z*ny + y)*nx + x; every boundary is periodic (Section 3).
 *
 * One step runs the method in its natural order, each stage a separate pass
 * over the whole grid, with no fusion:
 *   phi = sum_i f_i                                  Eq. order-parameter
 *   mu  = 4 beta (phi-phi_l)(phi-phi_v)(phi-phibar) - kappa lap(phi)
 *                                                    Eq. chemical_potencial
 *   grad(phi), grad(mu), lap(phi): isotropic stencils  Eqs. gradient, Laplace
 *   rho(phi), nu(phi) linear in phi                  Eq. vis and the text above it
 *   F = -phi grad(mu) + G_body                       Section 2.1, text after Eq. 6
 *   rho u = sum_i c_i g_i + F/2                      moments after Eq. GGi
 *   p = cs2/(1-w0) [sum_{i!=0} g_i + u.grad(rho)/2 + rho s_0(u)]
 *   f_i* = f_i - (f_i - f_i^eq)/tau_f + F_i + (1/2) d_t F_i   Eqs. BGK, H_i, F_i
 *   g_i* = g_i - (g_i - g_i^eq)/tau_g + G_i          Eqs. BGK-NS, G_i, Siu, GGi
 *   f_i(x + c_i, t+1) = f_i*(x), same for g          left-hand sides of BGK, BGK-NS
 *
 * Readings where the paper is silent, garbled or ambiguous:
 *   R1  (1/2) dt^2 d_t F_i is a backward difference in time, so the CH source
 *       is w_i b_i (1.5 S^n - 0.5 S^{n-1}) with S = u.grad(phi) and
 *       b_i = -1 + (|c_i|^2 - D cs2)/(2 cs2); S^{-1} = 0.
 *   R3  phi_l = 1 and phi_v = 0 by default; rho and nu are linear in
 *       (phi - phi_v)/(phi_l - phi_v), which is the paper's nu formula when
 *       phi_l = 1, phi_v = 0 (its "nu_g" is read as nu_v).
 *   R4  the last term of G_i is (u grad(rho)) : (c_i c_i - cs2 I) / cs2
 *       = [(c_i.u)(c_i.grad rho) - cs2 u.grad(rho)] / cs2.
 *   R5  cs = c/sqrt(3), so cs2 = 1/3 in lattice units (dx = dt = 1).
 *   R6  the D2Q9 velocities follow Eq. eq:ci in the paper's order, with the
 *       diagonal vectors scaled by sqrt(2) (the printed formula omits it).
 *   R7  grad(rho) = (rho_l - rho_v)/(phi_l - phi_v) grad_h(phi).
 *   R9  initial populations f = f^eq(phi0, mu(phi0)), g = 0 (p = 0, u = 0),
 *       S_prev = 0.
 *   D3Q19 is not in the paper; it uses the standard 19-velocity set, the
 *   same equilibria, sources and isotropic stencils with its own weights.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define WBO_QMAX 19

/* Coefficient of u.grad(rho) in the pressure recovery below Eq. GGi: the
 * paper's dt/2.  The oracle always uses dt/2; the tests rebuild it with
 * other values, on the CPU, only to show that their pins of this term fail
 * for a dropped, doubled or sign-flipped term. */
#ifndef WBO_P_UGR
#define WBO_P_UGR 0.5
#endif

/* ------------------------------------------------------------------ lattice */

typedef struct {
    int D, Q;
    int c[WBO_QMAX][3];
    double w[WBO_QMAX];
} wbo_lat;

static const double CS2 = 1.0 / 3.0; /* R5 */

/* D2Q9 of Eq. eq:ci (reading R6) and the weights given below Eq. H_iyang. */
static void lattice_d2q9(wbo_lat *L)
{
    const double pi = 3.14159265358979323846;
    memset(L, 0, sizeof *L);
    L->D = 2;
    L->Q = 9;
    L->w[0] = 4.0 / 9.0;
    for (int i = 1; i <= 4; ++i) {
        double th = (i - 2) * pi / 2.0;
        L->c[i][0] = (int)lround(cos(th));
        L->c[i][1] = (int)lround(sin(th));
        L->w[i] = 1.0 / 9.0;
    }
    for (int i = 5; i <= 8; ++i) {
        double th = (i - 5) * pi / 2.0 + pi / 4.0;
        L->c[i][0] = (int)lround(sqrt(2.0) * cos(th));
        L->c[i][1] = (int)lround(sqrt(2.0) * sin(th));
        L->w[i] = 1.0 / 36.0;
    }
}

/* Standard D3Q19 (not in the paper): rest, 6 face neighbours, 12 edges. */
static void lattice_d3q19(wbo_lat *L)
{
    memset(L, 0, sizeof *L);
    L->D = 3;
    L->Q = 19;
    L->w[0] = 1.0 / 3.0;
    int k = 1;
    for (int a = 0; a < 3; ++a)
        for (int s = 1; s >= -1; s -= 2) {
            L->c[k][a] = s;
            L->w[k] = 1.0 / 18.0;
            ++k;
        }
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            for (int sa = 1; sa >= -1; sa -= 2)
                for (int sb = 1; sb >= -1; sb -= 2) {
                    L->c[k][a] = sa;
                    L->c[k][b] = sb;
                    L->w[k] = 1.0 / 36.0;
                    ++k;
                }
}

static int lattice_make(int id, wbo_lat *L)
{
    if (id == 0) { lattice_d2q9(L); return 0; }
    if (id == 1) { lattice_d3q19(L); return 0; }
    return -1;
}

int wbo_lattice(int id, int *D, int *Q, int *c, double *w)
{
    wbo_lat L;
    if (lattice_make(id, &L)) return -1;
    *D = L.D;
    *Q = L.Q;
    for (int i = 0; i < L.Q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
        w[i] = L.w[i];
    }
    return 0;
}

/* --------------------------------------------------------------- parameters */

/* Parameter vector shared with the Python side (indices fixed). */
enum {
    P_W, P_M, P_ALPHA, P_SIGMA, P_PHIL, P_PHIV, P_RHOL, P_RHOV, P_NUL, P_NUV,
    P_GX, P_GY, P_GZ, P_TAUF, P_COUNT
};

typedef struct {
    double W, M, alpha, sigma, phil, phiv, rhol, rhov, nul, nuv, G[3];
    double kappa, beta, tauf;
} wbo_par;

/* Eq. beta gives beta = 8 kappa / (W^2 dphi^2) and Eq. suiface_tension gives
 * sigma = |dphi|^3 sqrt(2 kappa beta) / 6.  Substituting the first into the
 * second, sqrt(2 kappa beta) = 4 kappa / (W |dphi|), so
 * sigma = 2 kappa dphi^2 / (3 W):  kappa = 3 W sigma / (2 dphi^2) and
 * beta = 12 sigma / (W dphi^4). */
void wbo_kappa_beta(double W, double sigma, double phil, double phiv,
                    double *kappa, double *beta)
{
    double d2 = (phil - phiv) * (phil - phiv);
    *kappa = 3.0 * W * sigma / (2.0 * d2);
    *beta = 12.0 * sigma / (W * d2 * d2);
}

/* Eq. mobility: M = cs2 alpha (tau_f - 1/2) dt.  tau_f = 0 on input means
 * "derive tau_f from M and alpha"; otherwise alpha is derived from M, tau_f. */
static void params_make(const double *prm, wbo_par *P)
{
    P->W = prm[P_W];
    P->M = prm[P_M];
    P->alpha = prm[P_ALPHA];
    P->sigma = prm[P_SIGMA];
    P->phil = prm[P_PHIL];
    P->phiv = prm[P_PHIV];
    P->rhol = prm[P_RHOL];
    P->rhov = prm[P_RHOV];
    P->nul = prm[P_NUL];
    P->nuv = prm[P_NUV];
    P->G[0] = prm[P_GX];
    P->G[1] = prm[P_GY];
    P->G[2] = prm[P_GZ];
    wbo_kappa_beta(P->W, P->sigma, P->phil, P->phiv, &P->kappa, &P->beta);
    if (prm[P_TAUF] > 0.0) {
        P->tauf = prm[P_TAUF];
        P->alpha = P->M / (CS2 * (P->tauf - 0.5));
    } else {
        P->tauf = 0.5 + P->M / (CS2 * P->alpha);
    }
}

/* Eq. bulk_energy: psi(phi) = beta (phi - phi_l)^2 (phi - phi_v)^2. */
double wbo_psi(double beta, double phil, double phiv, double phi)
{
    return beta * (phi - phil) * (phi - phil) * (phi - phiv) * (phi - phiv);
}

/* d psi / d phi, the bulk part of Eq. chemical_potencial. */
double wbo_dpsi(double beta, double phil, double phiv, double phi)
{
    return 4.0 * beta * (phi - phil) * (phi - phiv) * (phi - 0.5 * (phil + phiv));
}

/* Linear interpolation between the phases ("a simple linear form as used for
 * density", Eq. vis; readings R3, R8). */
static double lin_phase(const wbo_par *P, double phi, double vl, double vv)
{
    return vv + (phi - P->phiv) / (P->phil - P->phiv) * (vl - vv);
}

/* ------------------------------------------------------ per-node components */

static double dot3(const int *c, const double *v, int D)
{
    double s = 0.0;
    for (int a = 0; a < D; ++a) s += c[a] * v[a];
    return s;
}

/* Eq. H_i: velocity-free CH equilibrium. */
static void feq_node(const wbo_lat *L, double phi, double mu, double alpha, double *out)
{
    out[0] = phi - (1.0 - L->w[0]) * alpha * mu;
    for (int i = 1; i < L->Q; ++i) out[i] = L->w[i] * alpha * mu;
}

/* Eq. F_i with S = u.grad(phi):
 * F_i = w_i S [-1 + I:(c_i c_i - cs2 I)/(2 cs2)],  I:(c c - cs2 I) = |c|^2 - D cs2. */
static void srcF_node(const wbo_lat *L, double S, double *out)
{
    for (int i = 0; i < L->Q; ++i) {
        double cc = 0.0;
        for (int a = 0; a < L->D; ++a) cc += (double)L->c[i][a] * L->c[i][a];
        double b = -1.0 + (cc - L->D * CS2) / (2.0 * CS2);
        out[i] = L->w[i] * S * b;
    }
}

/* Eq. Siu. */
static double s_node(const wbo_lat *L, int i, const double *u)
{
    double cu = dot3(L->c[i], u, L->D);
    double uu = 0.0;
    for (int a = 0; a < L->D; ++a) uu += u[a] * u[a];
    return L->w[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. G_i: pressure-based hydrodynamic equilibrium. */
static void geq_node(const wbo_lat *L, double p, double rho, const double *u, double *out)
{
    out[0] = p / CS2 * (L->w[0] - 1.0) + rho * s_node(L, 0, u);
    for (int i = 1; i < L->Q; ++i) out[i] = p / CS2 * L->w[i] + rho * s_node(L, i, u);
}

/* Eq. GGi with reading R4. */
static void forceG_node(const wbo_lat *L, double taug, const double *u,
                        const double *grho, const double *F, double *out)
{
    double ugr = 0.0;
    for (int a = 0; a < L->D; ++a) ugr += u[a] * grho[a];
    for (int i = 0; i < L->Q; ++i) {
        double cF = dot3(L->c[i], F, L->D);
        double cu = dot3(L->c[i], u, L->D);
        double cg = dot3(L->c[i], grho, L->D);
        double aniso = (cu * cg - CS2 * ugr) / CS2;
        out[i] = (1.0 - 1.0 / (2.0 * taug)) * L->w[i] * (ugr + cF / CS2 + aniso);
    }
}

/* Exported single-node forms, used by the moment-identity tests. */
int wbo_node_feq(int lat, double phi, double mu, double alpha, double *out)
{
    wbo_lat L;
    if (lattice_make(lat, &L)) return -1;
    feq_node(&L, phi, mu, alpha, out);
    return 0;
}

int wbo_node_F(int lat, double S, double *out)
{
    wbo_lat L;
    if (lattice_make(lat, &L)) return -1;
    srcF_node(&L, S, out);
    return 0;
}

int wbo_node_geq(int lat, double p, double rho, const double *u, double *out)
{
    wbo_lat L;
    if (lattice_make(lat, &L)) return -1;
    geq_node(&L, p, rho, u, out);
    return 0;
}

int wbo_node_G(int lat, double taug, const double *u, const double *grho,
               const double *F, double *out)
{
    wbo_lat L;
    if (lattice_make(lat, &L)) return -1;
    forceG_node(&L, taug, u, grho, F, out);
    return 0;
}

/* ---------------------------------------------------------------- the grid */

typedef struct wbo_sim {
    int nx, ny, nz, N;
    wbo_lat L;
    wbo_par P;
    long t;
    double *f, *g, *S_prev;              /* state at time t */
    /* work fields (recomputed every step) */
    double *phi, *mu, *lap, *gphi, *gmu, *u, *p, *rho, *S;
    double *fs, *gs;                     /* post-collision populations */
} wbo_sim;

/* Periodic neighbour x + c_i of node n. */
static int nbr(const wbo_sim *s, int n, const int *c)
{
    int x = n % s->nx, y = (n / s->nx) % s->ny, z = n / (s->nx * s->ny);
    x = (x + c[0] + s->nx) % s->nx;
    y = (y + c[1] + s->ny) % s->ny;
    z = (z + c[2] + s->nz) % s->nz;
    return (z * s->ny + y) * s->nx + x;
}

/* Eq. gradient: grad Psi(x) = sum_{i!=0} w_i c_i Psi(x + c_i) / (cs2 dt). */
static void field_grad(const wbo_sim *s, const double *psi, double *out)
{
    const wbo_lat *L = &s->L;
    for (int n = 0; n < s->N; ++n) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int i = 1; i < L->Q; ++i) {
            double v = psi[nbr(s, n, L->c[i])];
            for (int a = 0; a < L->D; ++a) acc[a] += L->w[i] * L->c[i][a] * v;
        }
        for (int a = 0; a < L->D; ++a) out[a * s->N + n] = acc[a] / CS2;
    }
}

/* Eq. Laplace: lap Psi(x) = sum_{i!=0} 2 w_i [Psi(x + c_i) - Psi(x)] / (cs2 dt^2). */
static void field_lap(const wbo_sim *s, const double *psi, double *out)
{
    const wbo_lat *L = &s->L;
    for (int n = 0; n < s->N; ++n) {
        double acc = 0.0;
        for (int i = 1; i < L->Q; ++i)
            acc += 2.0 * L->w[i] * (psi[nbr(s, n, L->c[i])] - psi[n]);
        out[n] = acc / CS2;
    }
}

/* Eq. chemical_potencial on the grid. */
static void field_mu(const wbo_sim *s, const double *phi, double *lap, double *mu)
{
    field_lap(s, phi, lap);
    for (int n = 0; n < s->N; ++n)
        mu[n] = wbo_dpsi(s->P.beta, s->P.phil, s->P.phiv, phi[n]) - s->P.kappa * lap[n];
}

wbo_sim *wbo_create(int nx, int ny, int nz, int lattice, const double *prm)
{
    if (nx < 1 || ny < 1 || nz < 1) return NULL;
    wbo_sim *s = (wbo_sim *)calloc(1, sizeof *s);
    if (!s) return NULL;
    if (lattice_make(lattice, &s->L)) { free(s); return NULL; }
    if (s->L.D == 2 && nz != 1) { free(s); return NULL; }
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->N = nx * ny * nz;
    params_make(prm, &s->P);
    size_t N = (size_t)s->N, Q = (size_t)s->L.Q;
    s->f = calloc(Q * N, sizeof(double));
    s->g = calloc(Q * N, sizeof(double));
    s->fs = calloc(Q * N, sizeof(double));
    s->gs = calloc(Q * N, sizeof(double));
    s->S_prev = calloc(N, sizeof(double));
    s->S = calloc(N, sizeof(double));
    s->phi = calloc(N, sizeof(double));
    s->mu = calloc(N, sizeof(double));
    s->lap = calloc(N, sizeof(double));
    s->rho = calloc(N, sizeof(double));
    s->p = calloc(N, sizeof(double));
    s->gphi = calloc(3 * N, sizeof(double));
    s->gmu = calloc(3 * N, sizeof(double));
    s->u = calloc(3 * N, sizeof(double));
    return s;
}

void wbo_destroy(wbo_sim *s)
{
    if (!s) return;
    double *bufs[] = {s->f, s->g, s->fs, s->gs, s->S_prev, s->S, s->phi, s->mu,
                      s->lap, s->rho, s->p, s->gphi, s->gmu, s->u};
    for (size_t k = 0; k < sizeof bufs / sizeof bufs[0]; ++k) free(bufs[k]);
    free(s);
}

/* kappa, beta, tau_f, alpha actually used. */
void wbo_derived(const wbo_sim *s, double *out)
{
    out[0] = s->P.kappa;
    out[1] = s->P.beta;
    out[2] = s->P.tauf;
    out[3] = s->P.alpha;
}

long wbo_time(const wbo_sim *s) { return s->t; }

/* Reading R9: f = f^eq(phi0, mu(phi0)), g = 0, S_prev = 0, t = 0. */
void wbo_init_phi(wbo_sim *s, const double *phi0)
{
    const int N = s->N, Q = s->L.Q;
    memcpy(s->phi, phi0, (size_t)N * sizeof(double));
    field_mu(s, s->phi, s->lap, s->mu);
    double fe[WBO_QMAX];
    for (int n = 0; n < N; ++n) {
        feq_node(&s->L, s->phi[n], s->mu[n], s->P.alpha, fe);
        for (int i = 0; i < Q; ++i) {
            s->f[i * N + n] = fe[i];
            s->g[i * N + n] = 0.0;
        }
        s->S_prev[n] = 0.0;
    }
    s->t = 0;
}

/* Macroscopic fields of the state at time t: phi, mu, grad(phi), grad(mu),
 * rho, F (kept implicit), u, p and S = u.grad(phi). */
static void compute_macros(wbo_sim *s)
{
    const wbo_lat *L = &s->L;
    const wbo_par *P = &s->P;
    const int N = s->N, Q = L->Q, D = L->D;

    /* Eq. order-parameter */
    for (int n = 0; n < N; ++n) {
        double acc = 0.0;
        for (int i = 0; i < Q; ++i) acc += s->f[i * N + n];
        s->phi[n] = acc;
    }
    /* Eq. chemical_potencial */
    field_mu(s, s->phi, s->lap, s->mu);
    /* Eq. gradient on phi and mu */
    field_grad(s, s->phi, s->gphi);
    field_grad(s, s->mu, s->gmu);

    const double drho = (P->rhol - P->rhov) / (P->phil - P->phiv);
    for (int n = 0; n < N; ++n) {
        double phi = s->phi[n];
        double rho = lin_phase(P, phi, P->rhol, P->rhov);
        double F[3] = {0.0, 0.0, 0.0}, grho[3] = {0.0, 0.0, 0.0}, u[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < D; ++a) {
            F[a] = -phi * s->gmu[a * N + n] + P->G[a];      /* F = F_s + G */
            grho[a] = drho * s->gphi[a * N + n];            /* R7 */
        }
        /* rho u = sum_i c_i g_i + 0.5 dt F */
        for (int a = 0; a < D; ++a) {
            double m = 0.0;
            for (int i = 0; i < Q; ++i) m += L->c[i][a] * s->g[i * N + n];
            u[a] = (m + 0.5 * F[a]) / rho;
        }
        /* p = cs2/(1 - w0) [sum_{i!=0} g_i + 0.5 dt u.grad(rho) + rho s_0(u)] */
        double sg = 0.0;
        for (int i = 1; i < Q; ++i) sg += s->g[i * N + n];
        double ugr = 0.0, ugp = 0.0;
        for (int a = 0; a < D; ++a) {
            ugr += u[a] * grho[a];
            ugp += u[a] * s->gphi[a * N + n];
        }
        s->p[n] = CS2 / (1.0 - L->w[0]) * (sg + WBO_P_UGR * ugr + rho * s_node(L, 0, u));
        s->rho[n] = rho;
        for (int a = 0; a < 3; ++a) s->u[a * N + n] = u[a];
        s->S[n] = ugp;                                       /* S = u.grad(phi) */
    }
}

static void collide(wbo_sim *s)
{
    const wbo_lat *L = &s->L;
    const wbo_par *P = &s->P;
    const int N = s->N, Q = L->Q, D = L->D;
    const double drho = (P->rhol - P->rhov) / (P->phil - P->phiv);
    double fe[WBO_QMAX], Fn[WBO_QMAX], Fo[WBO_QMAX], ge[WBO_QMAX], Gi[WBO_QMAX];
    for (int n = 0; n < N; ++n) {
        double phi = s->phi[n], rho = s->rho[n];
        double u[3] = {0.0, 0.0, 0.0}, F[3] = {0.0, 0.0, 0.0}, grho[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < D; ++a) {
            u[a] = s->u[a * N + n];
            F[a] = -phi * s->gmu[a * N + n] + P->G[a];
            grho[a] = drho * s->gphi[a * N + n];
        }
        /* CH population, Eq. BGK with Eqs. H_i and F_i; reading R1 for the
         * (1/2) dt^2 d_t F_i term: F_i^n + (F_i^n - F_i^{n-1})/2. */
        feq_node(L, phi, s->mu[n], P->alpha, fe);
        srcF_node(L, s->S[n], Fn);
        srcF_node(L, s->S_prev[n], Fo);
        for (int i = 0; i < Q; ++i) {
            double fi = s->f[i * N + n];
            s->fs[i * N + n] = fi - (fi - fe[i]) / P->tauf + Fn[i] + 0.5 * (Fn[i] - Fo[i]);
        }
        /* Hydrodynamic population, Eq. BGK-NS; nu(phi) linear (Eq. vis) and
         * nu = cs2 (tau_g - 1/2) dt. */
        double nu = lin_phase(P, phi, P->nul, P->nuv);
        double taug = 0.5 + nu / CS2;
        geq_node(L, s->p[n], rho, u, ge);
        forceG_node(L, taug, u, grho, F, Gi);
        for (int i = 0; i < Q; ++i) {
            double gi = s->g[i * N + n];
            s->gs[i * N + n] = gi - (gi - ge[i]) / taug + Gi[i];
        }
    }
}

/* f_i(x + c_i dt, t + dt) = f_i*(x, t): periodic streaming. */
static void stream(wbo_sim *s)
{
    const wbo_lat *L = &s->L;
    const int N = s->N;
    for (int i = 0; i < L->Q; ++i)
        for (int n = 0; n < N; ++n) {
            int m = nbr(s, n, L->c[i]);
            s->f[i * N + m] = s->fs[i * N + n];
            s->g[i * N + m] = s->gs[i * N + n];
        }
}

void wbo_step(wbo_sim *s, int nsteps)
{
    for (int k = 0; k < nsteps; ++k) {
        compute_macros(s);
        collide(s);
        stream(s);
        memcpy(s->S_prev, s->S, (size_t)s->N * sizeof(double));
        s->t += 1;
    }
}

/* Macroscopic fields at the current time t.  u has D*N entries ([a][n]). */
void wbo_macros(wbo_sim *s, double *phi, double *mu, double *p, double *u)
{
    compute_macros(s);
    const int N = s->N;
    if (phi) memcpy(phi, s->phi, (size_t)N * sizeof(double));
    if (mu) memcpy(mu, s->mu, (size_t)N * sizeof(double));
    if (p) memcpy(p, s->p, (size_t)N * sizeof(double));
    if (u) memcpy(u, s->u, (size_t)s->L.D * N * sizeof(double));
}

/* Diagnostics at time t: out = {sum phi, E = 1/2 sum rho |u|^2, max |u|,
 * min mu, max mu, sum (1.5 S - 0.5 S_prev)}.  The last entry is the exact
 * per-step phi budget: sum phi^{t+1} = sum phi^t - sum (1.5 S - 0.5 S_prev),
 * because sum_i f_i^eq = phi and sum_i F_i = -S (Eq. sumfeqandF). */
void wbo_diag(wbo_sim *s, double *out)
{
    compute_macros(s);
    const int N = s->N, D = s->L.D;
    double sphi = 0.0, E = 0.0, umax = 0.0, mumin = s->mu[0], mumax = s->mu[0], bud = 0.0;
    for (int n = 0; n < N; ++n) {
        double uu = 0.0;
        for (int a = 0; a < D; ++a) uu += s->u[a * N + n] * s->u[a * N + n];
        sphi += s->phi[n];
        E += 0.5 * s->rho[n] * uu;
        if (sqrt(uu) > umax) umax = sqrt(uu);
        if (s->mu[n] < mumin) mumin = s->mu[n];
        if (s->mu[n] > mumax) mumax = s->mu[n];
        bud += 1.5 * s->S[n] - 0.5 * s->S_prev[n];
    }
    out[0] = sphi;
    out[1] = E;
    out[2] = umax;
    out[3] = mumin;
    out[4] = mumax;
    out[5] = bud;
}

void wbo_get_state(const wbo_sim *s, double *f, double *g, double *S_prev)
{
    size_t QN = (size_t)s->L.Q * s->N;
    if (f) memcpy(f, s->f, QN * sizeof(double));
    if (g) memcpy(g, s->g, QN * sizeof(double));
    if (S_prev) memcpy(S_prev, s->S_prev, (size_t)s->N * sizeof(double));
}

void wbo_set_state(wbo_sim *s, const double *f, const double *g, const double *S_prev, long t)
{
    size_t QN = (size_t)s->L.Q * s->N;
    memcpy(s->f, f, QN * sizeof(double));
    memcpy(s->g, g, QN * sizeof(double));
    memcpy(s->S_prev, S_prev, (size_t)s->N * sizeof(double));
    s->t = t;
}

/* Stand-alone stencils on a caller field (for the stencil tests). */
void wbo_field_grad(const wbo_sim *s, const double *psi, double *out) { field_grad(s, psi, out); }
void wbo_field_lap(const wbo_sim *s, const double *psi, double *out) { field_lap(s, psi, out); }
void wbo_field_mu(const wbo_sim *s, const double *phi, double *out)
{
    double *lap = (double *)malloc((size_t)s->N * sizeof(double));
    field_mu(s, phi, lap, out);
    free(lap);
}

/* =====================================================================
 * Discrete adjoint (reverse mode) of the time step above, FP64.
 *
 * Not in the paper: the gradient of the discrete map, derived by
 * differentiating each stage of the step in reverse order.  It is pinned by
 * central finite differences of the forward map (tests), not by the paper.
 * Loss L(f^N, g^N, S^N); the adjoint of a state is (lf, lg, lS) =
 * (dL/df, dL/dg, dL/dS_prev) in the paper's convention.  Parameters: kappa,
 * beta (from sigma) and 1/tau_f (from M); their adjoints accumulate in
 * dpar = {dL/dkappa, dL/dbeta, dL/d(1/tau_f)}.
 * ===================================================================== */

/* d^2 psi / d phi^2 */
static double d2psi(const wbo_par *P, double phi)
{
    const double a = phi - P->phil, b = phi - P->phiv, c = phi - 0.5 * (P->phil + P->phiv);
    return 4.0 * P->beta * (b * c + a * c + a * b);
}

/* Transpose of the isotropic gradient (Eq. gradient): the stencil maps a
 * scalar psi to D components; its transpose maps D components v to
 * (G^T v)(y) = sum_i (w_i c_i / cs2) . v(y - c_i). */
static void field_grad_T(const wbo_sim *s, const double *v, double *out)
{
    const wbo_lat *L = &s->L;
    const int N = s->N;
    for (int n = 0; n < N; ++n) out[n] = 0.0;
    for (int x = 0; x < N; ++x)
        for (int i = 1; i < L->Q; ++i) {
            const int y = nbr(s, x, L->c[i]);  /* grad(x) reads psi(x + c_i) */
            double acc = 0.0;
            for (int a = 0; a < L->D; ++a) acc += L->w[i] * L->c[i][a] * v[a * N + x];
            out[y] += acc / CS2;
        }
}

/* Transpose of the Laplacian (Eq. Laplace): (L^T v)(y) = sum_x L(x, y) v(x). */
static void field_lap_T(const wbo_sim *s, const double *v, double *out)
{
    const wbo_lat *L = &s->L;
    const int N = s->N;
    for (int n = 0; n < N; ++n) out[n] = 0.0;
    for (int x = 0; x < N; ++x)
        for (int i = 1; i < L->Q; ++i) {
            const int y = nbr(s, x, L->c[i]);
            out[y] += 2.0 * L->w[i] * v[x] / CS2;
            out[x] -= 2.0 * L->w[i] * v[x] / CS2;
        }
}

/* One reverse step.  On entry s holds the state at time n (f, g, S_prev)
 * and (lf, lg, lS) the adjoint of the state at time n+1; on exit they hold
 * the adjoint of the state at time n.  dpar accumulates. */
static void adjoint_step(wbo_sim *s, double *lf, double *lg, double *lS, double *dpar)
{
    const wbo_lat *L = &s->L;
    const wbo_par *P = &s->P;
    const int N = s->N, Q = L->Q, D = L->D;
    compute_macros(s);  /* phi, mu, lap, grad phi, grad mu, rho, u, p, S of time n */
    const double drho = (P->rhol - P->rhov) / (P->phil - P->phiv);
    const double dnu = (P->nul - P->nuv) / (P->phil - P->phiv);
    const double itf = 1.0 / P->tauf;

    double *lfs = (double *)calloc((size_t)Q * N, sizeof(double));
    double *lgs = (double *)calloc((size_t)Q * N, sizeof(double));
    double *lphi = (double *)calloc((size_t)N, sizeof(double));
    double *lmu = (double *)calloc((size_t)N, sizeof(double));
    double *lgphi = (double *)calloc((size_t)3 * N, sizeof(double));
    double *lgmu = (double *)calloc((size_t)3 * N, sizeof(double));
    double *tmp = (double *)calloc((size_t)N, sizeof(double));
    double *lf_new = (double *)calloc((size_t)Q * N, sizeof(double));
    double *lg_new = (double *)calloc((size_t)Q * N, sizeof(double));
    double *lS_new = (double *)calloc((size_t)N, sizeof(double));

    /* reverse streaming: f_i(x + c_i, n+1) = f_i*(x) */
    for (int i = 0; i < Q; ++i)
        for (int x = 0; x < N; ++x) {
            const int y = nbr(s, x, L->c[i]);
            lfs[i * N + x] = lf[i * N + y];
            lgs[i * N + x] = lg[i * N + y];
        }

    double fe[WBO_QMAX], ge[WBO_QMAX];
    for (int x = 0; x < N; ++x) {
        const double phi = s->phi[x], mu = s->mu[x], rho = s->rho[x], p = s->p[x];
        double u[3] = {0, 0, 0}, F[3] = {0, 0, 0}, grho[3] = {0, 0, 0}, gph[3] = {0, 0, 0},
               gmu[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            u[a] = s->u[a * N + x];
            gph[a] = s->gphi[a * N + x];
            gmu[a] = s->gmu[a * N + x];
            F[a] = -phi * gmu[a] + P->G[a];
            grho[a] = drho * gph[a];
        }
        const double nu = lin_phase(P, phi, P->nul, P->nuv);
        const double taug = 0.5 + nu / CS2, itg = 1.0 / taug;
        double lu[3] = {0, 0, 0}, lF[3] = {0, 0, 0}, lgr[3] = {0, 0, 0}, lgp[3] = {0, 0, 0};
        double lrho = 0.0, lp = 0.0, lSx = 0.0, litg = 0.0, lph = 0.0, lmux = 0.0;

        /* CH collision: f* = (1 - 1/tau_f) f + f^eq/tau_f + w_i b_i (1.5 S - 0.5 S_prev) */
        feq_node(L, phi, mu, P->alpha, fe);
        double lsrc = 0.0;
        for (int i = 0; i < Q; ++i) {
            const double l = lfs[i * N + x];
            double cc = 0.0;
            for (int a = 0; a < D; ++a) cc += (double)L->c[i][a] * L->c[i][a];
            const double b = -1.0 + (cc - D * CS2) / (2.0 * CS2);
            lf_new[i * N + x] += (1.0 - itf) * l;
            dpar[2] += l * (fe[i] - s->f[i * N + x]);
            lsrc += l * L->w[i] * b;
            const double lfe = l * itf;  /* f^eq_0 = phi - (1-w0) alpha mu, f^eq_i = w_i alpha mu */
            if (i == 0) {
                lph += lfe;
                lmux += -(1.0 - L->w[0]) * P->alpha * lfe;
            } else {
                lmux += L->w[i] * P->alpha * lfe;
            }
        }
        lSx += 1.5 * lsrc;
        lS_new[x] += -0.5 * lsrc;  /* S_prev of time n */
        lSx += lS[x];               /* S_prev of time n+1 is S of time n */

        /* NS collision: g* = (1 - 1/tau_g) g + g^eq/tau_g + (1 - 1/(2 tau_g)) Gam_i,
         * Gam_i = w_i [u.grad rho + c.F/cs2 + ((c.u)(c.grad rho) - cs2 u.grad rho)/cs2] */
        geq_node(L, p, rho, u, ge);
        double ugr = 0.0, uu = 0.0;
        for (int a = 0; a < D; ++a) {
            ugr += u[a] * grho[a];
            uu += u[a] * u[a];
        }
        for (int i = 0; i < Q; ++i) {
            const double l = lgs[i * N + x];
            const double gi = s->g[i * N + x];
            double cF = 0, cu = 0, cg = 0;
            for (int a = 0; a < D; ++a) {
                cF += L->c[i][a] * F[a];
                cu += L->c[i][a] * u[a];
                cg += L->c[i][a] * grho[a];
            }
            const double gam = L->w[i] * (ugr + cF / CS2 + (cu * cg - CS2 * ugr) / CS2);
            lg_new[i * N + x] += (1.0 - itg) * l;
            litg += l * (ge[i] - gi) - 0.5 * l * gam;
            const double lge = l * itg, lgam = l * (1.0 - 0.5 * itg);
            /* g^eq_i = p/cs2 (w_i - delta_i0) + rho w_i [cu/cs2 + cu^2/(2 cs4) - uu/(2 cs2)] */
            lp += lge * (L->w[i] - (i == 0 ? 1.0 : 0.0)) / CS2;
            lrho += lge * L->w[i] * (cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2));
            for (int a = 0; a < D; ++a) {
                lu[a] += lge * rho * L->w[i] *
                         (L->c[i][a] / CS2 + cu * L->c[i][a] / (CS2 * CS2) - u[a] / CS2);
                /* Gam_i */
                lF[a] += lgam * L->w[i] * L->c[i][a] / CS2;
                lu[a] += lgam * L->w[i] * (grho[a] + (L->c[i][a] * cg - CS2 * grho[a]) / CS2);
                lgr[a] += lgam * L->w[i] * (u[a] + (cu * L->c[i][a] - CS2 * u[a]) / CS2);
            }
        }
        /* tau_g = 1/2 + nu(phi)/cs2 */
        lph += litg * (-(dnu / CS2) * itg * itg);

        /* S = u.grad phi */
        for (int a = 0; a < D; ++a) {
            lu[a] += lSx * gph[a];
            lgp[a] += lSx * u[a];
        }
        /* p = cs2/(1 - w0) [sum_{i!=0} g_i + u.grad rho / 2 + rho s_0(u)],
         * rho s_0 = -rho w0 uu / (2 cs2) */
        {
            const double k = CS2 / (1.0 - L->w[0]);
            for (int i = 1; i < Q; ++i) lg_new[i * N + x] += k * lp;
            for (int a = 0; a < D; ++a) {
                lu[a] += k * lp * (WBO_P_UGR * grho[a] - rho * L->w[0] * u[a] / CS2);
                lgr[a] += k * lp * WBO_P_UGR * u[a];
            }
            lrho += k * lp * (-L->w[0] * uu / (2 * CS2));
        }
        /* grad rho = drho grad phi */
        for (int a = 0; a < D; ++a) lgp[a] += drho * lgr[a];
        /* u = (sum c g + F/2) / rho */
        for (int a = 0; a < D; ++a) {
            const double lj = lu[a] / rho;
            for (int i = 0; i < Q; ++i) lg_new[i * N + x] += L->c[i][a] * lj;
            lF[a] += 0.5 * lj;
            lrho += -lu[a] * u[a] / rho;
        }
        /* F = -phi grad mu + G */
        for (int a = 0; a < D; ++a) {
            lph += -lF[a] * gmu[a];
            lgmu[a * N + x] += -phi * lF[a];
            lgphi[a * N + x] += lgp[a];
        }
        /* rho linear in phi */
        lph += drho * lrho;
        lphi[x] += lph;
        lmu[x] += lmux;
    }
    /* grad mu -> mu */
    field_grad_T(s, lgmu, tmp);
    for (int x = 0; x < N; ++x) lmu[x] += tmp[x];
    /* mu = dpsi(phi) - kappa lap(phi): parameters and phi */
    for (int x = 0; x < N; ++x) {
        dpar[0] += lmu[x] * (-s->lap[x]);
        dpar[1] += lmu[x] * wbo_dpsi(P->beta, P->phil, P->phiv, s->phi[x]) / P->beta;
        lphi[x] += d2psi(P, s->phi[x]) * lmu[x];
    }
    field_lap_T(s, lmu, tmp);
    for (int x = 0; x < N; ++x) lphi[x] += -P->kappa * tmp[x];
    field_grad_T(s, lgphi, tmp);
    for (int x = 0; x < N; ++x) lphi[x] += tmp[x];
    /* phi = sum_i f_i */
    for (int i = 0; i < Q; ++i)
        for (int x = 0; x < N; ++x) lf_new[i * N + x] += lphi[x];

    memcpy(lf, lf_new, (size_t)Q * N * sizeof(double));
    memcpy(lg, lg_new, (size_t)Q * N * sizeof(double));
    memcpy(lS, lS_new, (size_t)N * sizeof(double));
    double *bufs[] = {lfs, lgs, lphi, lmu, lgphi, lgmu, tmp, lf_new, lg_new, lS_new};
    for (size_t k = 0; k < sizeof bufs / sizeof bufs[0]; ++k) free(bufs[k]);
}

/* From the current state (time t0), run n steps forward keeping every state,
 * then propagate the adjoint (lf, lg, lS) of the final state back to time
 * t0, accumulating dpar.  The simulation is left at time t0 + n. */
void wbo_adjoint(wbo_sim *s, int n, double *lf, double *lg, double *lS, double *dpar)
{
    const size_t QN = (size_t)s->L.Q * s->N, N = (size_t)s->N;
    const size_t per = 2 * QN + N;
    double *hist = (double *)malloc((size_t)(n > 0 ? n : 1) * per * sizeof(double));
    for (int k = 0; k < n; ++k) {
        wbo_get_state(s, hist + k * per, hist + k * per + QN, hist + k * per + 2 * QN);
        wbo_step(s, 1);
    }
    double *fin = (double *)malloc(per * sizeof(double));
    wbo_get_state(s, fin, fin + QN, fin + 2 * QN);
    const long t_end = s->t;
    for (int k = n - 1; k >= 0; --k) {
        wbo_set_state(s, hist + k * per, hist + k * per + QN, hist + k * per + 2 * QN, t_end - n + k);
        adjoint_step(s, lf, lg, lS, dpar);
    }
    wbo_set_state(s, fin, fin + QN, fin + 2 * QN, t_end);
    free(fin);
    free(hist);
}

/* Adjoint of the initial condition (reading R9): f = f^eq(phi0, mu(phi0)),
 * g = 0, S_prev = 0.  Given lf at time 0, returns dL/dphi0 and adds the
 * kappa and beta contributions of mu(phi0) to dpar. */
void wbo_adjoint_init(wbo_sim *s, const double *phi0, const double *lf, double *lphi0, double *dpar)
{
    const wbo_lat *L = &s->L;
    const wbo_par *P = &s->P;
    const int N = s->N, Q = L->Q;
    double *mu = (double *)calloc((size_t)N, sizeof(double));
    double *lap = (double *)calloc((size_t)N, sizeof(double));
    double *lmu = (double *)calloc((size_t)N, sizeof(double));
    double *tmp = (double *)calloc((size_t)N, sizeof(double));
    field_mu(s, phi0, lap, mu);
    for (int x = 0; x < N; ++x) {
        lphi0[x] = lf[x];  /* f^eq_0 = phi - (1 - w0) alpha mu */
        double l = -(1.0 - L->w[0]) * P->alpha * lf[x];
        for (int i = 1; i < Q; ++i) l += L->w[i] * P->alpha * lf[i * N + x];
        lmu[x] = l;
        dpar[0] += l * (-lap[x]);
        dpar[1] += l * wbo_dpsi(P->beta, P->phil, P->phiv, phi0[x]) / P->beta;
        lphi0[x] += d2psi(P, phi0[x]) * l;
    }
    field_lap_T(s, lmu, tmp);
    for (int x = 0; x < N; ++x) lphi0[x] += -P->kappa * tmp[x];
    free(mu);
    free(lap);
    free(lmu);
    free(tmp);
}
