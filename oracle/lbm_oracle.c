/*
 * FP64 CPU oracle of the consistent two-phase lattice Boltzmann time step
 * of Zelko & Duenweg, "Consistent two-phase Lattice Boltzmann model for
 * gas-liquid systems" (arXiv:1402.2920).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of the method that the CUDA library is checked against.  Only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, table or helper with the CUDA library.
 *
 * Every lattice sweep of the supplemental step-by-step algorithm (steps 1-12
 * of the Supplemental Material, "S1".."S12" below) is a separate full pass
 * over the lattice, exactly as the supplement prescribes.  All arithmetic is
 * double precision.  Lattice units: h = a = 1 (captions of Tables I-III).
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   - Table I prints w0 of D3Q59 wrongly; the normalisation sum_i w_i = 1
 *     (Eq. tensor0_revised) forces w0 = 1 - 259/80 s + 273/64 s^2
 *     - 121/64 s^3, whose real root 1.1917145 is the c_s,max^2 the paper
 *     prints in Sec. III and App. B.
 *   - The c_s^2 in the j~ part of Xi' (S11) is c_s^2(rho0), as in Sec. VIII;
 *     only then is the third moment of Delta^corr equal to Xi.
 *   - "perm." in Xi' sums over the three choices of the lone index, applied
 *     to the whole brace.
 *   - The u-solve (S3-S7) stops when max_r max_a |j~new - j~| <= tol, and
 *     starts from the previous step's j~ when warm start is on (Sec. IX,
 *     item 3) or from zero (S1) otherwise.
 *   - Streaming is the push form of S11: n_new[i](r + c_i) = n_i(r) + Delta_i.
 *
 * Parity status: every function here is pinned by a test that does not
 * re-type its formula (weights: isotropy moments, printed c_s^2 window and
 * 3D->2D projection; equilibrium: its closed-form moments; stencils: Table
 * III moment conditions and exactness on polynomials; collision: the moment
 * identities of Secs. V, VI, VIII; the step: conservation, steady states,
 * the u-solve fixed point, the viscosities of Sec. VII, the linear
 * instability of the gas phase below the workloads' temperatures, and flat
 * slabs relaxing to the Maxwell coexistence densities of the van der Waals
 * and of App. B's psi-sine equations of state).  The Sigma and Xi' algebra of
 * S11 beyond what those identities fix is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXQ 59
#define MAXS 32
/* lattices smaller than this run single-threaded (thread start-up dominates) */
#define OMP_MIN_SITES 16384

/* lattice spacing and time step (captions of Tables I and II) */
static const double H = 1.0;
static const double A_LAT = 1.0;

/* ------------------------------------------------------------------------ */
/* Velocity sets and shells (Sec. III, Tables I and II)                      */
/* ------------------------------------------------------------------------ */

/* representative vector of every shell, in the order of the tables */
static const int REP3[8][3] = {{0,0,0},{1,0,0},{1,1,0},{1,1,1},{2,0,0},{2,2,0},{2,2,2},{4,0,0}};
static const int REP2[6][3] = {{0,0,0},{1,0,0},{1,1,0},{2,0,0},{2,2,0},{4,0,0}};

typedef struct {
    int d, Q, nshell;
    int c[MAXQ][3];
    int shell[MAXQ];
} orc_lattice;

/* All distinct vectors obtained from rep by permuting its first d components
 * and flipping signs, appended to out (deduplicated), +-pairs adjacent. */
static int expand_shell(const int rep[3], int d, int out[][3], int nout)
{
    static const int perm3[6][3] = {{0,1,2},{0,2,1},{1,0,2},{1,2,0},{2,0,1},{2,1,0}};
    static const int perm2[2][3] = {{0,1,2},{1,0,2}};
    const int (*perm)[3] = (d == 3) ? perm3 : perm2;
    int nperm = (d == 3) ? 6 : 2;
    int start = nout;
    for (int p = 0; p < nperm; ++p) {
        for (int sg = 0; sg < (1 << d); ++sg) {
            int v[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) {
                int comp = rep[perm[p][a]];
                v[a] = (sg >> a & 1) ? -comp : comp;
            }
            /* keep canonical member of each +- pair: first nonzero > 0 */
            int first = 0;
            for (int a = 0; a < d; ++a) if (v[a] != 0) { first = v[a]; break; }
            if (first < 0) continue;
            int dup = 0;
            for (int k = start; k < nout; ++k)
                if (out[k][0] == v[0] && out[k][1] == v[1] && out[k][2] == v[2]) dup = 1;
            if (dup) continue;
            out[nout][0] = v[0]; out[nout][1] = v[1]; out[nout][2] = v[2];
            ++nout;
            if (first != 0) {  /* its partner -c right after it */
                out[nout][0] = -v[0]; out[nout][1] = -v[1]; out[nout][2] = -v[2];
                ++nout;
            }
        }
    }
    return nout;
}

static void make_lattice(int lattice, orc_lattice* L)
{
    memset(L, 0, sizeof(*L));
    L->d = (lattice == 1) ? 3 : 2;
    L->nshell = (lattice == 1) ? 8 : 6;
    int n = 0;
    for (int s = 0; s < L->nshell; ++s) {
        const int* rep = (lattice == 1) ? REP3[s] : REP2[s];
        int n0 = n;
        n = expand_shell(rep, L->d, L->c, n);
        for (int k = n0; k < n; ++k) L->shell[k] = s;
    }
    L->Q = n;
}

/* Weight of shell k as a function of sigma2 = c_s^2.
 * D3Q59: Table I, with w0 corrected by normalisation (see header).
 * D2Q21: Table II as printed. */
static double weight_shell(int lattice, int k, double s)
{
    if (lattice == 1) {
        switch (k) {
        case 0: return 1.0 - 259.0/80.0*s + 273.0/64.0*s*s - 121.0/64.0*s*s*s;
        case 1: return 2.0*s*(8.0/45.0 - s/3.0 + s*s/6.0);
        case 2: return s*(8.0/45.0 - s/3.0 + s*s/6.0);
        case 3: return s/12.0*(-16.0/15.0 + 4.0*s - 2.5*s*s);
        case 4: return s/96.0*(-24.0/5.0 + 17.0*s - 9.0*s*s);
        case 5: return s/192.0*(-8.0/15.0 + s + s*s);
        case 6: return s/192.0*(4.0/15.0 - s + s*s);
        case 7: return s/384.0*(4.0/15.0 - s + s*s);
        }
    } else {
        switch (k) {
        case 0: return 1.0 - 22.5*s*(7.0/60.0 - 7.0/48.0*s + s*s/16.0);
        case 1: return s/3.0*(32.0/15.0 - 4.0*s + 2.0*s*s);
        case 2: return s*(s/3.0 - s*s/4.0);
        case 3: return s*(-1.0/18.0 + 3.0/16.0*s - s*s/12.0);
        case 4: return s/96.0*(-0.5*s + 1.5*s*s);
        case 5: return s/384.0*(4.0/15.0 - s + s*s);
        }
    }
    return NAN;
}

/* ------------------------------------------------------------------------ */
/* Finite-difference stencils (Sec. IV, Table III)                           */
/* ------------------------------------------------------------------------ */

enum { ST_D1 = 0, ST_LAP = 1, ST_TRACELESS = 2, ST_D3 = 3 };

typedef struct { int n; int d[MAXS][3]; double tau[MAXS]; } orc_stencil;

/* Table III columns; shells (0), (1 0), (1 1), (2 0) in both dimensions */
static double table3_tau(int d, int which, int shell)
{
    static const double t2[4][4] = {
        /* d/da      lap     traceless  d^3 */
        {0.0,        -4.0,   0.0,       0.0},   /* (00)  */
        {2.0/3.0,    1.0,    1.0,       -2.0},  /* (10)  */
        {0.0,        0.0,    0.25,      0.5},   /* (11)  */
        {-1.0/24.0,  0.0,    0.0,       0.25}}; /* (20)  */
    static const double t3[4][4] = {
        {0.0,        -6.0,   0.0,       0.0},   /* (000) */
        {2.0/3.0,    1.0,    0.5,       -3.0},  /* (100) */
        {0.0,        0.0,    0.25,      0.5},   /* (110) */
        {-1.0/24.0,  0.0,    0.0,       0.25}}; /* (200) */
    return (d == 3) ? t3[shell][which] : t2[shell][which];
}

static void make_stencil(int d, int which, orc_stencil* S)
{
    static const int reps[4][3] = {{0,0,0},{1,0,0},{1,1,0},{2,0,0}};
    int vec[MAXQ][3];
    S->n = 0;
    for (int sh = 0; sh < 4; ++sh) {
        double tau = table3_tau(d, which, sh);
        if (tau == 0.0) continue;  /* a zero coefficient contributes nothing */
        int m = expand_shell(reps[sh], d, vec, 0);
        for (int k = 0; k < m; ++k) {
            S->d[S->n][0] = vec[k][0]; S->d[S->n][1] = vec[k][1]; S->d[S->n][2] = vec[k][2];
            S->tau[S->n] = tau;
            ++S->n;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Equation of state (App. B; S1)                                            */
/* ------------------------------------------------------------------------ */

enum { EOS_VDW = 0, EOS_PSI_SINE = 1 };

typedef struct {
    int kind;
    double a, b, T;                  /* p = rho T / (1 - b rho) - a rho^2 */
    double rho1, rho2, A, cs2_1;     /* psi-sine construction of App. B     */
} orc_eos;

/* p, dp/drho, p - rho dp/drho, rho d2p/drho2 (the four items of S1) */
static void eos_eval(const orc_eos* e, double rho, double out[4])
{
    double p, dp, d2p;
    if (e->kind == EOS_VDW) {
        double g = 1.0 - e->b * rho;
        p = rho * e->T / g - e->a * rho * rho;
        dp = e->T / (g * g) - 2.0 * e->a * rho;
        d2p = 2.0 * e->b * e->T / (g * g * g) - 2.0 * e->a;
    } else {
        /* c_s^2(rho) = c_s^2(rho1) exp(int_{rho1}^{rho} psi), psi the sine
         * bump on (rho1, rho3), rho3 = 2 rho2 - rho1; p = rho c_s^2. */
        double D = e->rho2 - e->rho1;
        double rho3 = 2.0 * e->rho2 - e->rho1;
        double psi = 0.0, dpsi = 0.0, integral = 0.0;
        if (rho > e->rho1 && rho < rho3) {
            double ph = M_PI * (rho - e->rho1) / D;
            psi = e->A * sin(ph);
            dpsi = e->A * M_PI / D * cos(ph);
            integral = e->A * D / M_PI * (1.0 - cos(ph));
        }
        double cs2 = e->cs2_1 * exp(integral);
        p = rho * cs2;
        /* d(cs2)/drho = cs2 psi */
        dp = cs2 + rho * cs2 * psi;
        d2p = cs2 * psi * (1.0 + rho * psi) + cs2 * (psi + rho * dpsi);
    }
    out[0] = p;
    out[1] = dp;
    out[2] = p - rho * dp;
    out[3] = rho * d2p;
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int lattice;
    orc_lattice L;
    orc_stencil d1, d3;
    int nx, ny, nz;
    long N;
    orc_eos eos;
    double gamma, kappa, rho0, cs0;  /* cs0 = c_s^2(rho0) */
    double w0[MAXQ];                 /* w_i(rho0) */
    double tol;
    int maxit, warm;
    /* populations (pre-collision) and the new lattice of S11 */
    double *n, *nnew;
    /* fields, component-major [comp][N]; vectors have 3, tensors 9, 3-tensors 27 */
    double *rho, *j0, *p, *dp, *pm, *rpp, *f, *j0p, *jt, *jtn, *u, *j, *q, *du;
    double *dj, *dpg, *dpuu, *dpr, *Sig, *Xi;
    double *dA, *dB, *dC;
    /* diagnostics of the last u-solve */
    int last_iters;
    double last_resid;
    int converged;
} orc_sim;

static inline long site(const orc_sim* s, int x, int y, int z)
{
    return (long)x + (long)s->nx * ((long)y + (long)s->ny * (long)z);
}

static inline int wrap(int v, int n)
{
    int m = v % n;
    return m < 0 ? m + n : m;
}

static inline long neighbour(const orc_sim* s, long r, int dx, int dy, int dz)
{
    int x = (int)(r % s->nx);
    int y = (int)((r / s->nx) % s->ny);
    int z = (int)(r / ((long)s->nx * s->ny));
    return site(s, wrap(x + dx, s->nx), wrap(y + dy, s->ny), wrap(z + dz, s->nz));
}

/* A scalar field evaluated at a site: the argument of a lattice derivative. */
typedef double (*site_fn)(const orc_sim*, long r, int i, int k);

/* Sec. IV.B: (1/a) sum_i tau_i d_ia g(r + a d_i) */
static double D1(const orc_sim* s, long r, int a, site_fn g, int i, int k)
{
    double acc = 0.0;
    for (int m = 0; m < s->d1.n; ++m) {
        if (s->d1.d[m][a] == 0) continue;
        long rn = neighbour(s, r, s->d1.d[m][0], s->d1.d[m][1], s->d1.d[m][2]);
        acc += s->d1.tau[m] * s->d1.d[m][a] * g(s, rn, i, k);
    }
    return acc / A_LAT;
}

#define F3(arr, a, r) (s->arr[(long)(a) * s->N + (r)])
#define F9(arr, a, b, r) (s->arr[((long)(a) * 3 + (b)) * s->N + (r)])
#define F27(arr, a, b, c, r) (s->arr[(((long)(a) * 3 + (b)) * 3 + (c)) * s->N + (r)])

static double g_u(const orc_sim* s, long r, int i, int k) { (void)k; return F3(u, i, r); }
static double g_j(const orc_sim* s, long r, int i, int k) { (void)k; return F3(j, i, r); }
static double g_p(const orc_sim* s, long r, int i, int k) { (void)i; (void)k; return s->p[r]; }
static double g_q(const orc_sim* s, long r, int i, int k) { return F9(q, i, k, r); }
static double g_puu(const orc_sim* s, long r, int i, int k) { return s->p[r] * F3(u, i, r) * F3(u, k, r); }
static double g_pr(const orc_sim* s, long r, int i, int k) { (void)i; (void)k; return s->p[r] / s->rho[r]; }

static double div_u(const orc_sim* s, long r)
{
    double t = 0.0;
    for (int g = 0; g < s->L.d; ++g) t += F9(du, g, g, r);
    return t;
}
/* (p - rho p') d_g u_g  -- argument of the first derivative list of S11 */
static double g_A(const orc_sim* s, long r, int i, int k) { (void)i; (void)k; return s->pm[r] * div_u(s, r); }
/* p (d_a u_b + d_b u_a) */
static double g_B(const orc_sim* s, long r, int a, int b)
{
    return s->p[r] * (F9(du, a, b, r) + F9(du, b, a, r));
}
/* rho^-1 d_b p + u_g d_g u_b */
static double g_C(const orc_sim* s, long r, int b, int k)
{
    (void)k;
    double t = F3(dpg, b, r) / s->rho[r];
    for (int g = 0; g < s->L.d; ++g) t += F3(u, g, r) * F9(du, g, b, r);
    return t;
}

/* ------------------------------------------------------------------------ */
/* Equilibrium (Eq. equilibrium, Sec. III)                                   */
/* ------------------------------------------------------------------------ */

static double n_eq(const orc_sim* s, int i, double rho, double cs2, const double u[3])
{
    double w = weight_shell(s->lattice, s->L.shell[i], cs2);
    double uc = 0.0, uu = 0.0;
    for (int a = 0; a < s->L.d; ++a) { uc += u[a] * s->L.c[i][a]; uu += u[a] * u[a]; }
    return w * rho * (1.0 + uc / cs2 + uc * uc / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
}

/* ------------------------------------------------------------------------ */
/* The steps of the supplemental algorithm                                   */
/* ------------------------------------------------------------------------ */

/* S1: j~ reset (unless warm start), rho, j0, and the EOS items */
static void s1(orc_sim* s)
{
    const int d = s->L.d, Q = s->L.Q;
#pragma omp parallel for schedule(static) if (s->N >= OMP_MIN_SITES)
    for (long r = 0; r < s->N; ++r) {
        if (!s->warm)
            for (int a = 0; a < 3; ++a) F3(jt, a, r) = 0.0;
        double rho = 0.0, j0[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            double ni = s->n[(long)i * s->N + r];
            rho += ni;
            for (int a = 0; a < d; ++a) j0[a] += ni * s->L.c[i][a];
        }
        s->rho[r] = rho;
        for (int a = 0; a < 3; ++a) F3(j0, a, r) = j0[a];
        double e[4];
        eos_eval(&s->eos, rho, e);
        s->p[r] = e[0]; s->dp[r] = e[1]; s->pm[r] = e[2]; s->rpp[r] = e[3];
    }
}

/* S2: interface force f_a = kappa rho d_a d_b d_b rho (Sec. IV.E, Sec. VI)
 * and j0' = j0 + (h/2) f */
static void s2(orc_sim* s)
{
    const int d = s->L.d;
#pragma omp parallel for schedule(static) if (s->N >= OMP_MIN_SITES)
    for (long r = 0; r < s->N; ++r) {
        for (int a = 0; a < 3; ++a) {
            double acc = 0.0;
            if (a < d)
                for (int m = 0; m < s->d3.n; ++m) {
                    long rn = neighbour(s, r, s->d3.d[m][0], s->d3.d[m][1], s->d3.d[m][2]);
                    acc += s->d3.tau[m] * s->d3.d[m][a] * s->rho[rn];
                }
            F3(f, a, r) = s->kappa * s->rho[r] * acc / (A_LAT * A_LAT * A_LAT);
            F3(j0p, a, r) = F3(j0, a, r) + 0.5 * H * F3(f, a, r);
        }
    }
}

/* S3: u = rho^-1 (j0' + j~) */
static void s3(orc_sim* s)
{
#pragma omp parallel for schedule(static) if (s->N >= OMP_MIN_SITES)
    for (long r = 0; r < s->N; ++r)
        for (int a = 0; a < 3; ++a) F3(u, a, r) = (F3(j0p, a, r) + F3(jt, a, r)) / s->rho[r];
}

/* S4: d_a u_b (Sec. IV.B) and q_ab = (p - rho p') delta_ab d_g u_g + p (d_b u_a + d_a u_b) */
static void s4(orc_sim* s)
{
    const int d = s->L.d;
#pragma omp parallel for schedule(static) if (s->N >= OMP_MIN_SITES)
    for (long r = 0; r < s->N; ++r)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                F9(du, a, b, r) = (a < d && b < d) ? D1(s, r, a, g_u, b, 0) : 0.0;
#pragma omp parallel for schedule(static) if (s->N >= OMP_MIN_SITES)
    for (long r = 0; r < s->N; ++r) {
        double dv = div_u(s, r);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                F9(q, a, b, r) = (a < d && b < d)
                    ? s->pm[r] * (a == b ? 1.0 : 0.0) * dv + s->p[r] * (F9(du, b, a, r) + F9(du, a, b, r))
                    : 0.0;
    }
}

/* S5: j~new_a = -(h^2/12) d_b q_ab ; S6: the max-norm change */
static double s5_s6(orc_sim* s)
{
    const int d = s->L.d;
    double resid = 0.0;
#pragma omp parallel for schedule(static) reduction(max:resid) if (s->N >= OMP_MIN_SITES)
    for (long r = 0; r < s->N; ++r) {
        for (int a = 0; a < 3; ++a) {
            double acc = 0.0;
            if (a < d)
                for (int b = 0; b < d; ++b) acc += D1(s, r, b, g_q, a, b);
            double v = -(H * H / 12.0) * acc;
            F3(jtn, a, r) = v;
            double dlt = fabs(v - F3(jt, a, r));
            if (!(dlt <= resid)) resid = dlt;  /* NaN propagates */
        }
    }
    return resid;
}

/* S3-S8: the implicit u-solve (Sec. IX) */
static void usolve(orc_sim* s)
{
    int it = 0;
    double resid = INFINITY;
    s->converged = 0;
    for (;;) {
        s3(s);
        s4(s);
        resid = s5_s6(s);
        ++it;
        /* S7 / S8: j~ = j~new in either case */
        memcpy(s->jt, s->jtn, sizeof(double) * 3 * s->N);
        if (resid <= s->tol) { s->converged = 1; break; }
        if (it >= s->maxit || !isfinite(resid)) break;
    }
    s->last_iters = it;
    s->last_resid = resid;
    /* S8: j = j0' + j~, u = j / rho */
#pragma omp parallel for schedule(static) if (s->N >= OMP_MIN_SITES)
    for (long r = 0; r < s->N; ++r)
        for (int a = 0; a < 3; ++a) {
            F3(j, a, r) = F3(j0p, a, r) + F3(jt, a, r);
            F3(u, a, r) = F3(j, a, r) / s->rho[r];
        }
}

/* S10: first-order lattice derivatives of u, j, p, p u_b u_g, p/rho */
static void s10(orc_sim* s)
{
    const int d = s->L.d;
#pragma omp parallel for schedule(static) if (s->N >= OMP_MIN_SITES)
    for (long r = 0; r < s->N; ++r) {
        for (int a = 0; a < 3; ++a) {
            int ia = a < d;
            for (int b = 0; b < 3; ++b) {
                int ib = ia && b < d;
                F9(du, a, b, r) = ib ? D1(s, r, a, g_u, b, 0) : 0.0;
                F9(dj, a, b, r) = ib ? D1(s, r, a, g_j, b, 0) : 0.0;
                for (int c = 0; c < 3; ++c)
                    F27(dpuu, a, b, c, r) = (ib && c < d) ? D1(s, r, a, g_puu, b, c) : 0.0;
            }
            F3(dpg, a, r) = ia ? D1(s, r, a, g_p, 0, 0) : 0.0;
            F3(dpr, a, r) = ia ? D1(s, r, a, g_pr, 0, 0) : 0.0;
        }
    }
}

/* S11, first part at one site: the derivatives of the three bracketed
 * expressions, then Sigma_ab and Xi'_abc. */
static void s11_tensors(orc_sim* s, long r)
{
    const int d = s->L.d;
    const double g = s->gamma;
    for (int a = 0; a < 3; ++a) {
        F3(dA, a, r) = a < d ? D1(s, r, a, g_A, 0, 0) : 0.0;
        for (int b = 0; b < 3; ++b) {
            F9(dC, a, b, r) = (a < d && b < d) ? D1(s, r, a, g_C, b, 0) : 0.0;
            for (int c = 0; c < 3; ++c)   /* dB[g][a][b] = d_g [p (d_a u_b + d_b u_a)] */
                F27(dB, a, b, c, r) = (a < d && b < d && c < d) ? D1(s, r, a, g_B, b, c) : 0.0;
        }
    }
    double divu = div_u(s, r), divj = 0.0;
    for (int c = 0; c < d; ++c) divj += F9(dj, c, c, r);
    double trdC = 0.0;
    for (int c = 0; c < d; ++c) trdC += F9(dC, c, c, r);
    const double p = s->p[r], dp = s->dp[r], pm = s->pm[r], rpp = s->rpp[r];
    const double k1 = -(H * H / 4.0) * (g + 1.0) * (g + 1.0) / (g - 1.0);
    const double k2 = (H * H / 6.0) * (g * g + 4.0 * g + 1.0) / (g - 1.0);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double v = 0.0;
            if (a < d && b < d) {
                double ua = F3(u, a, r), ub = F3(u, b, r);
                double divBa = 0.0, divBb = 0.0;   /* d_g [p (d_a u_g + d_g u_a)] */
                for (int c = 0; c < d; ++c) { divBa += F27(dB, c, a, c, r); divBb += F27(dB, c, b, c, r); }
                double t1 = ua * F3(dA, b, r) + ub * F3(dA, a, r) + ub * divBa + ua * divBb;
                double dl = (a == b) ? 1.0 : 0.0;
                double t2 = -dp * divj * (F9(du, a, b, r) + F9(du, b, a, r))
                          - p * F9(dC, a, b, r) - p * F9(dC, b, a, r)
                          - pm * dl * trdC
                          + rpp * dl * divu * divj;
                v = k1 * t1 + k2 * t2;
            }
            F9(Sig, a, b, r) = v;
        }
    const double k3 = (H / 3.0) * (g * g + 4.0 * g + 1.0) / (g + 1.0);
    /* X(a,b;c) = d_c(p u_a u_b) + delta_ab [p d_c(p/rho) + (p - rho p') u_c d_e u_e] */
#define XT(A_, B_, C_) (F27(dpuu, C_, A_, B_, r) + ((A_) == (B_) ? (p * F3(dpr, C_, r) + pm * F3(u, C_, r) * divu) : 0.0))
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) {
                double v = 0.0;
                if (a < d && b < d && c < d) {
                    v = k3 * (XT(a, b, c) + XT(a, c, b) + XT(b, c, a));
                    v += (1.0 - g) * s->cs0 * ((a == b ? F3(jt, c, r) : 0.0) + (a == c ? F3(jt, b, r) : 0.0)
                                               + (b == c ? F3(jt, a, r) : 0.0));
                }
                F27(Xi, a, b, c, r) = v;
            }
#undef XT
}

/* S11, second part at one site: the three collision operators per velocity.
 * parts (optional) receives Delta^bulk, Delta^int, Delta^corr as [3][Q]. */
static void s11_collide(const orc_sim* s, long r, double* nstar, double* parts)
{
    const int d = s->L.d, Q = s->L.Q;
    const double g = s->gamma, c0 = s->cs0;
    const double rho = s->rho[r];
    const double cs2 = s->p[r] / rho;  /* local c_s^2 = p / rho */
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = F3(u, a, r);
    for (int i = 0; i < Q; ++i) {
        const int* c = s->L.c[i];
        double ni = s->n[(long)i * s->N + r];
        double neq = n_eq(s, i, rho, cs2, u);
        double dbulk = (g - 1.0) * (ni - neq);
        double cf = 0.0, cj = 0.0;
        for (int a = 0; a < d; ++a) { cf += c[a] * F3(f, a, r); cj += c[a] * F3(jt, a, r); }
        double dint = 0.5 * (1.0 + g) * H * s->w0[i] / c0 * cf;
        double h2 = 0.0, h3 = 0.0;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                double dab = (a == b) ? 1.0 : 0.0;
                h2 += F9(Sig, a, b, r) * (c[a] * c[b] - c0 * dab);
                for (int cc = 0; cc < d; ++cc) {
                    double dac = (a == cc) ? 1.0 : 0.0, dbc = (b == cc) ? 1.0 : 0.0;
                    h3 += F27(Xi, a, b, cc, r)
                        * ((double)c[a] * c[b] * c[cc] - c0 * (dab * c[cc] + dac * c[b] + dbc * c[a]));
                }
            }
        double dcorr = (g - 1.0) * s->w0[i] / c0 * cj
                     + s->w0[i] / (2.0 * c0 * c0) * h2
                     + s->w0[i] / (6.0 * c0 * c0 * c0) * h3;
        nstar[i] = ni + dbulk + dint + dcorr;
        if (parts) { parts[i] = dbulk; parts[Q + i] = dint; parts[2 * Q + i] = dcorr; }
    }
}

/* S11 sweep with push streaming into the new lattice */
static void s11(orc_sim* s)
{
    const int Q = s->L.Q;
#pragma omp parallel for schedule(static) if (s->N >= OMP_MIN_SITES)
    for (long r = 0; r < s->N; ++r) s11_tensors(s, r);
#pragma omp parallel for schedule(static) if (s->N >= OMP_MIN_SITES)
    for (long r = 0; r < s->N; ++r) {
        double nstar[MAXQ];
        s11_collide(s, r, nstar, NULL);
        for (int i = 0; i < Q; ++i) {
            long rn = neighbour(s, r, s->L.c[i][0], s->L.c[i][1], s->L.c[i][2]);
            s->nnew[(long)i * s->N + rn] = nstar[i];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Exported interface (ctypes)                                               */
/* ------------------------------------------------------------------------ */

int orc_lattice_info(int lattice, int* c_out, int* shell_out)
{
    orc_lattice L;
    make_lattice(lattice, &L);
    for (int i = 0; i < L.Q; ++i) {
        if (c_out) for (int a = 0; a < 3; ++a) c_out[3 * i + a] = L.c[i][a];
        if (shell_out) shell_out[i] = L.shell[i];
    }
    return L.Q;
}

void orc_weights(int lattice, double cs2, double* w_out)
{
    orc_lattice L;
    make_lattice(lattice, &L);
    for (int i = 0; i < L.Q; ++i) w_out[i] = weight_shell(lattice, L.shell[i], cs2);
}

double orc_weight_shell(int lattice, int shell, double cs2) { return weight_shell(lattice, shell, cs2); }

void orc_eos_eval(int kind, const double* prm /* a,b,T,rho1,rho2,A,cs2_1 */, double rho, double* out4)
{
    orc_eos e = {kind, prm[0], prm[1], prm[2], prm[3], prm[4], prm[5], prm[6]};
    eos_eval(&e, rho, out4);
}

/* stencil table: returns count, fills d (n*3) and tau (n) */
int orc_stencil_info(int d, int which, int* d_out, double* tau_out)
{
    orc_stencil S;
    make_stencil(d, which, &S);
    for (int m = 0; m < S.n; ++m) {
        for (int a = 0; a < 3; ++a) d_out[3 * m + a] = S.d[m][a];
        tau_out[m] = S.tau[m];
    }
    return S.n;
}

void orc_destroy(orc_sim* s);

orc_sim* orc_create(int lattice, int nx, int ny, int nz, int eos_kind, const double* eos_prm,
                    double gamma, double kappa, double rho0, double tol, int maxit, int warm)
{
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->lattice = lattice;
    make_lattice(lattice, &s->L);
    make_stencil(s->L.d, ST_D1, &s->d1);
    make_stencil(s->L.d, ST_D3, &s->d3);
    s->nx = nx; s->ny = ny; s->nz = (s->L.d == 2) ? 1 : nz;
    s->N = (long)s->nx * s->ny * s->nz;
    s->eos.kind = eos_kind;
    s->eos.a = eos_prm[0]; s->eos.b = eos_prm[1]; s->eos.T = eos_prm[2];
    s->eos.rho1 = eos_prm[3]; s->eos.rho2 = eos_prm[4]; s->eos.A = eos_prm[5]; s->eos.cs2_1 = eos_prm[6];
    s->gamma = gamma; s->kappa = kappa; s->rho0 = rho0;
    double e0[4];
    eos_eval(&s->eos, rho0, e0);
    s->cs0 = e0[0] / rho0;
    for (int i = 0; i < s->L.Q; ++i) s->w0[i] = weight_shell(lattice, s->L.shell[i], s->cs0);
    s->tol = tol; s->maxit = maxit; s->warm = warm;
    long N = s->N, Q = s->L.Q;
    double** one[] = {&s->rho, &s->p, &s->dp, &s->pm, &s->rpp};
    for (unsigned k = 0; k < sizeof(one) / sizeof(one[0]); ++k) *one[k] = (double*)calloc(N, sizeof(double));
    double** three[] = {&s->j0, &s->f, &s->j0p, &s->jt, &s->jtn, &s->u, &s->j, &s->dpg, &s->dpr, &s->dA};
    for (unsigned k = 0; k < sizeof(three) / sizeof(three[0]); ++k) *three[k] = (double*)calloc(3 * N, sizeof(double));
    double** nine[] = {&s->q, &s->du, &s->dj, &s->Sig, &s->dC};
    for (unsigned k = 0; k < sizeof(nine) / sizeof(nine[0]); ++k) *nine[k] = (double*)calloc(9 * N, sizeof(double));
    s->dpuu = (double*)calloc(27 * N, sizeof(double));
    s->Xi = (double*)calloc(27 * N, sizeof(double));
    s->dB = (double*)calloc(27 * N, sizeof(double));
    s->n = (double*)calloc(Q * N, sizeof(double));
    s->nnew = (double*)calloc(Q * N, sizeof(double));
    if (!s->n || !s->nnew || !s->dB || !s->Xi || !s->dpuu || !s->q || !s->Sig || !s->rho || !s->jt) {
        orc_destroy(s);
        return NULL;
    }
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    double* all[] = {s->n, s->nnew, s->rho, s->j0, s->p, s->dp, s->pm, s->rpp, s->f, s->j0p, s->jt, s->jtn,
                     s->u, s->j, s->q, s->du, s->dj, s->dpg, s->dpuu, s->dpr, s->Sig, s->Xi, s->dA, s->dB, s->dC};
    for (unsigned k = 0; k < sizeof(all) / sizeof(all[0]); ++k) free(all[k]);
    free(s);
}

int orc_Q(const orc_sim* s) { return s->L.Q; }
double orc_cs0(const orc_sim* s) { return s->cs0; }

/* Initial condition: n_i = n_i^eq(rho, u) with the local c_s^2 = p/rho, and
 * j~ = 0 (the paper is silent on the start; this is the design's reading). */
void orc_init(orc_sim* s, const double* rho, const double* u /* 3*N or NULL */)
{
    for (long r = 0; r < s->N; ++r) {
        double e[4];
        eos_eval(&s->eos, rho[r], e);
        double cs2 = e[0] / rho[r];
        double uu[3] = {0.0, 0.0, 0.0};
        if (u) for (int a = 0; a < s->L.d; ++a) uu[a] = u[(long)a * s->N + r];
        for (int i = 0; i < s->L.Q; ++i) s->n[(long)i * s->N + r] = n_eq(s, i, rho[r], cs2, uu);
        for (int a = 0; a < 3; ++a) F3(jt, a, r) = 0.0;
    }
}

/* One or more full time steps (S1..S12).  Returns 0, or -4 if a u-solve did
 * not reach tol within maxit sweeps (the step is still completed). */
int orc_step(orc_sim* s, int nsteps)
{
    int status = 0;
    for (int t = 0; t < nsteps; ++t) {
        s1(s);
        s2(s);
        usolve(s);
        if (!s->converged) status = -4;
        s10(s);
        s11(s);
        /* S12: rename n_new to n */
        double* tmp = s->n; s->n = s->nnew; s->nnew = tmp;
    }
    return status;
}

/* S1-S8 on the current populations without collision: rho and u = j/rho.
 * The warm-start j~ of the simulation is left as it was. */
int orc_fields(orc_sim* s, double* rho, double* u)
{
    double* save = (double*)malloc(sizeof(double) * 3 * s->N);
    if (!save) return -5;
    memcpy(save, s->jt, sizeof(double) * 3 * s->N);
    s1(s);
    s2(s);
    usolve(s);
    if (rho) memcpy(rho, s->rho, sizeof(double) * s->N);
    if (u) memcpy(u, s->u, sizeof(double) * 3 * s->N);
    memcpy(s->jt, save, sizeof(double) * 3 * s->N);
    free(save);
    return s->converged ? 0 : -4;
}

void orc_get_pops(const orc_sim* s, double* out) { memcpy(out, s->n, sizeof(double) * s->L.Q * s->N); }
void orc_set_pops(orc_sim* s, const double* in) { memcpy(s->n, in, sizeof(double) * s->L.Q * s->N); }
void orc_get_jt(const orc_sim* s, double* out) { memcpy(out, s->jt, sizeof(double) * 3 * s->N); }
int orc_last_iters(const orc_sim* s) { return s->last_iters; }
double orc_last_resid(const orc_sim* s) { return s->last_resid; }

/* Fields of the most recent step, by name, for the identity tests. */
int orc_field(const orc_sim* s, const char* name, double* out)
{
    struct { const char* nm; double* ptr; long ncomp; } tab[] = {
        {"rho", s->rho, 1}, {"j0", s->j0, 3}, {"p", s->p, 1}, {"dp", s->dp, 1}, {"pm", s->pm, 1},
        {"rpp", s->rpp, 1}, {"f", s->f, 3}, {"j0p", s->j0p, 3}, {"jt", s->jt, 3}, {"u", s->u, 3},
        {"j", s->j, 3}, {"du", s->du, 9}, {"dj", s->dj, 9}, {"dp_grad", s->dpg, 3}, {"dpuu", s->dpuu, 27},
        {"dpr", s->dpr, 3}, {"Sigma", s->Sig, 9}, {"Xi", s->Xi, 27}, {"q", s->q, 9}};
    for (unsigned k = 0; k < sizeof(tab) / sizeof(tab[0]); ++k)
        if (strcmp(tab[k].nm, name) == 0) {
            memcpy(out, tab[k].ptr, sizeof(double) * tab[k].ncomp * s->N);
            return (int)tab[k].ncomp;
        }
    return -1;
}

/* S1, S2, S3-S8, S10 and the tensors of S11 on the current populations,
 * without collision or streaming: leaves every field of the step in place
 * so that the per-site collision can be examined with orc_collision_parts. */
int orc_prepare(orc_sim* s)
{
    s1(s);
    s2(s);
    usolve(s);
    s10(s);
#pragma omp parallel for schedule(static) if (s->N >= OMP_MIN_SITES)
    for (long r = 0; r < s->N; ++r) s11_tensors(s, r);
    return s->converged ? 0 : -4;
}

/* Delta^bulk, Delta^int, Delta^corr at site r as [3][Q] (after orc_prepare) */
void orc_collision_parts(const orc_sim* s, long r, double* parts, double* nstar)
{
    double tmp[MAXQ];
    s11_collide(s, r, nstar ? nstar : tmp, parts);
}

/* The lattice derivative operators of Table III applied to a periodic
 * scalar field g (nx*ny*nz).  which: 0 first derivative (out: 3*N),
 * 1 Laplacian (out: N), 2 traceless second derivative (out: 9*N),
 * 3 third derivative d_a d_b d_b (out: 3*N). */
void orc_apply_stencil(int d, int which, int nx, int ny, int nz, const double* g, double* out)
{
    orc_stencil S;
    make_stencil(d, which, &S);
    orc_sim tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.nx = nx; tmp.ny = ny; tmp.nz = (d == 2) ? 1 : nz;
    tmp.N = (long)tmp.nx * tmp.ny * tmp.nz;
    const long N = tmp.N;
    for (long r = 0; r < N; ++r) {
        if (which == ST_LAP) {
            double acc = 0.0;
            for (int m = 0; m < S.n; ++m) acc += S.tau[m] * g[neighbour(&tmp, r, S.d[m][0], S.d[m][1], S.d[m][2])];
            out[r] = acc;
        } else if (which == ST_TRACELESS) {
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double acc = 0.0;
                    if (a < d && b < d)
                        for (int m = 0; m < S.n; ++m) {
                            double dd = 0.0;
                            for (int c = 0; c < d; ++c) dd += (double)S.d[m][c] * S.d[m][c];
                            double t = (double)S.d[m][a] * S.d[m][b] - (a == b ? dd / d : 0.0);
                            acc += S.tau[m] * t * g[neighbour(&tmp, r, S.d[m][0], S.d[m][1], S.d[m][2])];
                        }
                    out[(long)(a * 3 + b) * N + r] = acc;
                }
        } else {
            for (int a = 0; a < 3; ++a) {
                double acc = 0.0;
                if (a < d)
                    for (int m = 0; m < S.n; ++m)
                        acc += S.tau[m] * S.d[m][a] * g[neighbour(&tmp, r, S.d[m][0], S.d[m][1], S.d[m][2])];
                out[(long)a * N + r] = acc;
            }
        }
    }
}

/* equilibrium populations at one state point (for the moment tests) */
void orc_neq(int lattice, double rho, double cs2, const double* u3, double* out)
{
    orc_sim tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.lattice = lattice;
    make_lattice(lattice, &tmp.L);
    for (int i = 0; i < tmp.L.Q; ++i) out[i] = n_eq(&tmp, i, rho, cs2, u3);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
