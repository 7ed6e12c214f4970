/*
 * FP64 CPU oracle of the relaxing-TVD ideal-MHD update of Wong, Wong, Feng & Tang,
 * "Efficient magnetohydrodynamic simulations on graphics processing units with CUDA"
 * (arXiv:0908.4362), Sect. 3 (numerical scheme) and Sect. 4.2 (program flow).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct reference
 * that the CUDA path is compared against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code with the CUDA path.
 *
 * Conventions (where the paper is silent, the reading taken is stated beside the code):
 *   - 8 fields per cell, f[0..7] = (rho, rho vx, rho vy, rho vz, E, Bx, By, Bz), Sect. 4.1.
 *   - Flat index (x*ny + y)*nz + z, z contiguous (Sect. 4.1, index equations).
 *   - B is face-centred (Eq. "equat_b"): Bx[i] lives on the x-face i-1/2, By[j] on y-face
 *     j-1/2, Bz[k] on z-face k-1/2.  Cell width h on all axes (the paper uses h = 1).
 *   - Local sweep coordinates for axis a: normal n = a, transverse t1 = (a+1)%3,
 *     t2 = (a+2)%3.  Every sweep is written once, in local coordinates.
 *   - Boundaries per axis: periodic (wrap) or outflow (clamp every array index to
 *     [0, N-1], i.e. zero-gradient ghosts).  The paper does not discuss boundaries.
 *   - Everything in double precision, compiled with -ffp-contract=off (no FMA).
 *
 * Status bits returned by the sweeps: 1 = unphysical (rho <= 0 or a negative fast-speed
 * radicand), 2 = non-finite value produced.  Computation continues, as in the method.
 *
 * ORC_MUTANT (compile-time, default 0) plants one known mistake at a time; the test suite
 * builds those variants to show that its pins catch each of them.  Production builds of
 * the oracle always have ORC_MUTANT == 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

typedef struct {
    int n[3];      /* nx, ny, nz (each >= 1) */
    int bc[3];     /* 0 = periodic, 1 = outflow */
    double h;      /* cell width */
    double gamma;  /* ratio of specific heats */
    double cfl;    /* Courant number */
} orc_grid;

enum { ORC_UNPHYSICAL = 1, ORC_NONFINITE = 2 };

int orc_mutant(void) { return ORC_MUTANT; }

/* ------------------------------------------------------------------------------------ */
/* index helpers                                                                         */
/* ------------------------------------------------------------------------------------ */

static int imap(int i, int n, int bc)
{
    if (bc == 0) {
        i %= n;
        if (i < 0) i += n;
        return i;
    }
    if (i < 0) return 0;
    if (i >= n) return n - 1;
    return i;
}

static long flat(const orc_grid* g, const int c[3])
{
    return ((long)c[0] * g->n[1] + c[1]) * g->n[2] + c[2];
}

/* global coordinates of (position i along axis a, p along t1, q along t2), each mapped */
static long at_local(const orc_grid* g, int a, int i, int p, int q)
{
    int t1 = (a + 1) % 3, t2 = (a + 2) % 3, c[3];
    c[a] = imap(i, g->n[a], g->bc[a]);
    c[t1] = imap(p, g->n[t1], g->bc[t1]);
    c[t2] = imap(q, g->n[t2], g->bc[t2]);
    return flat(g, c);
}

/* ------------------------------------------------------------------------------------ */
/* van Leer limiter, Eq. "eq:limiter": 2ab/(a+b); no correction when the two one-sided   */
/* corrections have opposite signs (text before Eq. "eq:Delta_F_n"), extended to ab = 0. */
/* ------------------------------------------------------------------------------------ */

double orc_vanleer(double a, double b)
{
#if ORC_MUTANT == 4
    return 0.5 * (a + b);                 /* mistake: unlimited central correction */
#else
    double ab = a * b;
    if (ab > 0.0) return 2.0 * ab / (a + b);
    return 0.0;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* Cell flux in local coordinates, Eqs. "eq:flux", "eq:lr" and the freezing speed of     */
/* Sect. 3 (text before Eq. "equat_CFL").                                                */
/*   u = (rho, m_n, m_t1, m_t2, E), b = cell-centred (B_n, B_t1, B_t2).                   */
/*   Returns fr = (c u + F)/2, fl = (c u - F)/2: the fluxes c u^R and c u^L of the        */
/*   right- and left-moving variables u^{R,L} = (u +- F/c)/2.                             */
/* ------------------------------------------------------------------------------------ */

int orc_cell_flux(const double* u, const double* b, double gamma,
                  double* fr, double* fl, double* c_out, double* F_out)
{
    int st = 0;
    double rho = u[0];
    double vn = u[1] / rho, vt1 = u[2] / rho, vt2 = u[3] / rho;
    double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    double v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
#if ORC_MUTANT == 7
    double p = (gamma - 1.0) * (u[4] - 0.5 * rho * v2);   /* mistake: B^2/2 dropped */
#else
    double p = (gamma - 1.0) * (u[4] - 0.5 * rho * v2 - 0.5 * b2);
#endif
    double ps = p + 0.5 * b2;                              /* P* = p + B^2/2 */
    double bv = b[0] * vn + b[1] * vt1 + b[2] * vt2;
    double F[5];
    F[0] = u[1];
    F[1] = u[1] * vn + ps - b[0] * b[0];
#if ORC_MUTANT == 1
    F[2] = u[2] * vn;                                      /* mistake: -B_n B_t1 dropped */
#else
    F[2] = u[2] * vn - b[0] * b[1];
#endif
    F[3] = u[3] * vn - b[0] * b[2];
    F[4] = (u[4] + ps) * vn - b[0] * bv;
    double rad = gamma * p / rho + b2 / rho;
#if ORC_MUTANT == 8
    rad = gamma * p / rho;                                 /* mistake: B^2/rho dropped */
#endif
    if (!(rho > 0.0) || rad < 0.0) st |= ORC_UNPHYSICAL;
    double c = fabs(vn) + sqrt(rad);
    for (int k = 0; k < 5; ++k) {
        fr[k] = 0.5 * (c * u[k] + F[k]);
        fl[k] = 0.5 * (c * u[k] - F[k]);
        if (F_out) F_out[k] = F[k];
    }
    if (c_out) *c_out = c;
    return st;
}

/* ------------------------------------------------------------------------------------ */
/* fluid_a(dt): Algorithm 1 with Eqs. "eq:Delta_u_half" and "eq:Delta_u_full".            */
/* B is held fixed and interpolated to cell centres (Algorithm 1, step 3).                */
/* ------------------------------------------------------------------------------------ */

#define FG 3   /* ghost cells each side of a fluid pencil */

static int fluid_pencil(const orc_grid* g, double* const f[8], int a, int p, int q,
                        double dt, double* w)
{
    const int N = g->n[a], L = N + 2 * FG;
    const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    const double dth = dt / g->h;
    double* u   = w;            /* L x 5 */
    double* bc  = u + 5 * L;    /* L x 3 */
    double* fr  = bc + 3 * L;   /* L x 5 */
    double* fl  = fr + 5 * L;
    double* uh  = fl + 5 * L;   /* L x 5, u^{t+dt/2} */
    double* g1  = uh + 5 * L;   /* L x 5, first-order interface flux at i+1/2 */
    double* g2  = g1 + 5 * L;   /* L x 5, second-order interface flux at i+1/2 */
    int st = 0;
    const int fld[5] = {0, 1 + a, 1 + t1, 1 + t2, 4};

    for (int e = 0; e < L; ++e) {
        int i = e - FG;
        long c = at_local(g, a, i, p, q);
        for (int k = 0; k < 5; ++k) u[5 * e + k] = f[fld[k]][c];
        /* face averages to the cell centre; the neighbour face is mapped on its own axis */
        long cn = at_local(g, a, i + 1, p, q);
        long c1 = at_local(g, a, i, p + 1, q);
        long c2 = at_local(g, a, i, p, q + 1);
        bc[3 * e + 0] = 0.5 * (f[5 + a][c] + f[5 + a][cn]);
        bc[3 * e + 1] = 0.5 * (f[5 + t1][c] + f[5 + t1][c1]);
        bc[3 * e + 2] = 0.5 * (f[5 + t2][c] + f[5 + t2][c2]);
    }
    /* stage 1: first-order upwind fluxes from u^t */
    for (int e = 0; e < L; ++e)
        st |= orc_cell_flux(u + 5 * e, bc + 3 * e, g->gamma, fr + 5 * e, fl + 5 * e, 0, 0);
    for (int e = 0; e + 1 < L; ++e)          /* interface e+1/2 */
        for (int k = 0; k < 5; ++k) g1[5 * e + k] = fr[5 * e + k] - fl[5 * (e + 1) + k];
#if ORC_MUTANT == 13
    const double half = 1.0;                 /* mistake: predictor over a full dt */
#else
    const double half = 0.5;
#endif
    for (int e = 1; e + 1 < L; ++e)
        for (int k = 0; k < 5; ++k)
            uh[5 * e + k] = u[5 * e + k] - half * dth * (g1[5 * e + k] - g1[5 * (e - 1) + k]);
    /* stage 2: van Leer limited fluxes from u^{t+dt/2} */
    for (int e = 1; e + 1 < L; ++e)
        st |= orc_cell_flux(uh + 5 * e, bc + 3 * e, g->gamma, fr + 5 * e, fl + 5 * e, 0, 0);
    for (int e = 2; e + 3 < L; ++e) {        /* interface e+1/2 needs cells e-1 .. e+2 */
        for (int k = 0; k < 5; ++k) {
            double frm = fr[5 * (e - 1) + k], fr0 = fr[5 * e + k], frp = fr[5 * (e + 1) + k];
            double fl0 = fl[5 * e + k], fl1 = fl[5 * (e + 1) + k], fl2 = fl[5 * (e + 2) + k];
            /* right-moving: F_n + phi((F_n - F_{n-1})/2, (F_{n+1} - F_n)/2), Eq. "eq:F_n" */
            double right = fr0 + orc_vanleer(0.5 * (fr0 - frm), 0.5 * (frp - fr0));
            /* left-moving: mirror image, upwind cell is e+1 */
#if ORC_MUTANT == 5
            double left = fl1 + orc_vanleer(0.5 * (fl1 - fl0), 0.5 * (fl2 - fl1));  /* sign */
#else
            double left = fl1 - orc_vanleer(0.5 * (fl1 - fl0), 0.5 * (fl2 - fl1));
#endif
            g2[5 * e + k] = right - left;
        }
    }
    /* full update and scatter (pencils along a never overlap) */
    for (int e = FG; e < FG + N; ++e) {
        long c = at_local(g, a, e - FG, p, q);
        for (int k = 0; k < 5; ++k) {
            double un = u[5 * e + k] - dth * (g2[5 * e + k] - g2[5 * (e - 1) + k]);
            if (!isfinite(un)) st |= ORC_NONFINITE;
            f[fld[k]][c] = un;
        }
        if (!(f[0][c] > 0.0)) st |= ORC_UNPHYSICAL;
    }
    return st;
}

int orc_fluid(const orc_grid* g, double* const f[8], int a, double dt)
{
    const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    const int P = g->n[t1], Q = g->n[t2];
    const int L = g->n[a] + 2 * FG;
    int st = 0;
#pragma omp parallel reduction(| : st)
    {
        double* w = (double*)malloc(sizeof(double) * 38 * (size_t)L);
#pragma omp for collapse(2) schedule(static)
        for (int p = 0; p < P; ++p)
            for (int q = 0; q < Q; ++q) st |= fluid_pencil(g, f, a, p, q, dt, w);
        free(w);
    }
    return st;
}

/* ------------------------------------------------------------------------------------ */
/* CT_{t->a}(dt): advection of the transverse face field B_t along a, and the constraint  */
/* update of B_a with the same EMF (Sect. 3, Eqs. "eq:averaging_x", "eq:first_flux";      */
/* Algorithm 2).  The fluid is frozen at its post-fluid_a state.                          */
/* EMF layout: em[r * (N+1) + i] = EMF at the a-face i-1/2 of transverse row r, i=0..N.   */
/* ------------------------------------------------------------------------------------ */

#define CG 4   /* ghost cells each side of a CT pencil */

static void emf_pencil(const orc_grid* g, double* const f[8], int a, int tsel, int p, int q,
                       double dt, double* w, double* em)
{
    const int N = g->n[a], L = N + 2 * CG;
    const int t = (a + tsel) % 3;
    const double dth = dt / g->h;
    double* vf = w;          /* face velocity at the t-face, before smoothing */
    double* vs = vf + L;     /* smoothed along a, Eq. "eq:averaging_x" */
    double* bt = vs + L;
    double* e1 = bt + L;     /* first-order EMF at a-face e+1/2 */
    double* bh = e1 + L;     /* B_t at t + dt/2 */
    double* gg = bh + L;     /* v B at t + dt/2 */
    int pm = p - (tsel == 1), qm = q - (tsel == 2);   /* the cell across the t-face */

    for (int e = 0; e < L; ++e) {
        int i = e - CG;
        long c0 = at_local(g, a, i, p, q), c1 = at_local(g, a, i, pm, qm);
#if ORC_MUTANT == 6
        long c2 = at_local(g, a, i, p + (tsel == 1), q + (tsel == 2));  /* mistake: wrong side */
        vf[e] = (f[1 + a][c0] + f[1 + a][c1]) / (f[0][c0] + f[0][c2]);
#else
        vf[e] = (f[1 + a][c0] + f[1 + a][c1]) / (f[0][c0] + f[0][c1]);
#endif
        bt[e] = f[5 + t][c0];
    }
    /* (1,2,1)/4 with the two outer neighbours added first: the sum is then exactly odd
     * under a reflection of the a-axis (v_a -> -v_a, neighbours swapped), so the edge
     * velocity at a mirror face is exactly 0 and Eq. "eq:first_flux"'s rule decides it */
#if ORC_MUTANT == 14
    for (int e = 1; e + 1 < L; ++e) vs[e] = 0.25 * (vf[e + 1] + 2.0 * vf[e] + vf[e - 1]);  /* mistake: one-sided order */
#else
    for (int e = 1; e + 1 < L; ++e) vs[e] = 0.25 * ((vf[e + 1] + vf[e - 1]) + 2.0 * vf[e]);
#endif
    /* first-order upwind EMF by the sign of the edge velocity, Eq. "eq:first_flux" */
    for (int e = 1; e + 2 < L; ++e) {
        double ve = 0.5 * (vs[e] + vs[e + 1]);
        e1[e] = (ve > 0.0) ? vs[e] * bt[e] : vs[e + 1] * bt[e + 1];
    }
    for (int e = 2; e + 2 < L; ++e) {
        bh[e] = bt[e] - 0.5 * dth * (e1[e] - e1[e - 1]);
        gg[e] = vs[e] * bh[e];
    }
    /* second-order EMF: same relaxing-TVD correction and limiter as the fluid */
    for (int e = CG - 1; e < CG + N; ++e) {          /* a-faces -1/2 .. N-1/2 */
        double ve = 0.5 * (vs[e] + vs[e + 1]);
        double val;
        if (ve > 0.0)
            val = gg[e] + orc_vanleer(0.5 * (gg[e] - gg[e - 1]), 0.5 * (gg[e + 1] - gg[e]));
        else
            val = gg[e + 1] - orc_vanleer(0.5 * (gg[e + 1] - gg[e]), 0.5 * (gg[e + 2] - gg[e + 1]));
        em[e - (CG - 1)] = val;
    }
}

static int ct_one(const orc_grid* g, double* const f[8], int a, int tsel, double dt)
{
    const int t1 = (a + 1) % 3, t2 = (a + 2) % 3, t = (a + tsel) % 3;
    const int N = g->n[a], P = g->n[t1], Q = g->n[t2], L = N + 2 * CG;
    const double dth = dt / g->h;
    double* em = (double*)malloc(sizeof(double) * (size_t)P * Q * (N + 1));
    int st = 0;
#pragma omp parallel
    {
        double* w = (double*)malloc(sizeof(double) * 6 * (size_t)L);
#pragma omp for collapse(2) schedule(static)
        for (int p = 0; p < P; ++p)
            for (int q = 0; q < Q; ++q)
                emf_pencil(g, f, a, tsel, p, q, dt, w, em + ((long)p * Q + q) * (N + 1));
        free(w);
    }
    /* advection of B_t and constraint on B_a from the same EMF */
#pragma omp parallel for collapse(2) schedule(static) reduction(| : st)
    for (int p = 0; p < P; ++p)
        for (int q = 0; q < Q; ++q) {
            const double* e0 = em + ((long)p * Q + q) * (N + 1);
            int pn = p, qn = q;
#if ORC_MUTANT == 3
            if (tsel == 1) pn = imap(p - 1, P, g->bc[t1]); else qn = imap(q - 1, Q, g->bc[t2]);
#else
            if (tsel == 1) pn = imap(p + 1, P, g->bc[t1]); else qn = imap(q + 1, Q, g->bc[t2]);
#endif
            const double* en = em + ((long)pn * Q + qn) * (N + 1);
            for (int i = 0; i < N; ++i) {
                long c = at_local(g, a, i, p, q);
#if ORC_MUTANT == 2
                f[5 + t][c] += dth * (e0[i + 1] - e0[i]);    /* mistake: sign */
#else
                f[5 + t][c] -= dth * (e0[i + 1] - e0[i]);
#endif
                f[5 + a][c] += dth * (en[i] - e0[i]);
                if (!isfinite(f[5 + t][c]) || !isfinite(f[5 + a][c])) st |= ORC_NONFINITE;
            }
        }
    free(em);
    return st;
}

/* CT_{t1->a} followed by CT_{t2->a} (Algorithm 2, both halves). */
int orc_ct(const orc_grid* g, double* const f[8], int a, double dt)
{
    int st = ct_one(g, f, a, 1, dt);
    st |= ct_one(g, f, a, 2, dt);
    return st;
}

int orc_ct_one(const orc_grid* g, double* const f[8], int a, int tsel, double dt)
{
    return ct_one(g, f, a, tsel, dt);
}

/* ------------------------------------------------------------------------------------ */
/* CFL, Eq. "equat_CFL": c_max = max over cells of max(|vx|,|vy|,|vz|) +                  */
/* sqrt(gamma p/rho + B^2/rho) with cell-centred B.  The three squares in |v|^2 and |B|^2 */
/* are summed smallest first, so that c_max does not depend on the order of the axes.    */
/* ------------------------------------------------------------------------------------ */

static double sum3_sorted(double a, double b, double c)
{
    double t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    return (a + b) + c;
}

double orc_cell_cmax(const orc_grid* g, double* const f[8], long idx, int x, int y, int z,
                     int* st)
{
    int c[3] = {x, y, z};
    double bcen[3];
    for (int a = 0; a < 3; ++a) {
        int cn[3] = {x, y, z};
        cn[a] = imap(c[a] + 1, g->n[a], g->bc[a]);
        bcen[a] = 0.5 * (f[5 + a][idx] + f[5 + a][flat(g, cn)]);
    }
    double rho = f[0][idx];
    double vx = f[1][idx] / rho, vy = f[2][idx] / rho, vz = f[3][idx] / rho;
    double v2 = sum3_sorted(vx * vx, vy * vy, vz * vz);
    double b2 = sum3_sorted(bcen[0] * bcen[0], bcen[1] * bcen[1], bcen[2] * bcen[2]);
    double p = (g->gamma - 1.0) * (f[4][idx] - 0.5 * rho * v2 - 0.5 * b2);
    double rad = g->gamma * p / rho + b2 / rho;
    if (!(rho > 0.0) || rad < 0.0) *st |= ORC_UNPHYSICAL;
    double vm = fabs(vx);
    if (fabs(vy) > vm) vm = fabs(vy);
    if (fabs(vz) > vm) vm = fabs(vz);
    return vm + sqrt(rad);
}

double orc_cmax(const orc_grid* g, double* const f[8], int* status)
{
    double cm = 0.0;
    int st = 0;
#pragma omp parallel for collapse(2) reduction(max : cm) reduction(| : st) schedule(static)
    for (int x = 0; x < g->n[0]; ++x)
        for (int y = 0; y < g->n[1]; ++y)
            for (int z = 0; z < g->n[2]; ++z) {
                int c[3] = {x, y, z};
                double v = orc_cell_cmax(g, f, flat(g, c), x, y, z, &st);
                if (v > cm || v != v) cm = (v != v) ? INFINITY : v;
            }
    if (status) *status |= st;
    return cm;
}

/* ------------------------------------------------------------------------------------ */
/* One step: forward sweep L_c L_b L_a then reverse sweep L_a L_b L_c with the axis       */
/* order (a,b,c) cycled over three steps, Eq. "eq:L_sequence".  Forward L = fluid then    */
/* CT; reverse L = CT then fluid (end of Sect. 4.3).  All six L-ops use the same dt and   */
/* the step advances t by 2 dt (Sect. 4.2, step 8).                                        */
/* ------------------------------------------------------------------------------------ */

static const int ORDER[3][3] = {{0, 1, 2}, {2, 0, 1}, {1, 2, 0}};

int orc_step_dt(const orc_grid* g, double* const f[8], int phase, double dt)
{
    int st = 0;
    const int* o = ORDER[phase % 3];
#if ORC_MUTANT == 9
    o = ORDER[0];                             /* mistake: no cycling of the axis order */
#endif
    for (int k = 0; k < 3; ++k) {
        st |= orc_fluid(g, f, o[k], dt);
        st |= orc_ct(g, f, o[k], dt);
    }
    for (int k = 2; k >= 0; --k) {
#if ORC_MUTANT == 10
        st |= orc_fluid(g, f, o[k], dt);      /* mistake: reverse L not reversed */
        st |= orc_ct(g, f, o[k], dt);
#else
        st |= orc_ct(g, f, o[k], dt);
        st |= orc_fluid(g, f, o[k], dt);
#endif
    }
    return st;
}

/* dt from the CFL condition, scaled by the cell width and clipped to land on t_end
 * (t_end < 0: no end time).  Returns 0 when no step should be taken. */
double orc_dt(const orc_grid* g, double* const f[8], double t, double t_end, int* clipped,
              int* status)
{
    double cm = orc_cmax(g, f, status);
#if ORC_MUTANT == 11
    double dt = g->cfl / cm;                  /* mistake: cell width ignored */
#else
    double dt = g->cfl * g->h / cm;
#endif
    *clipped = 0;
    if (t_end >= 0.0) {
        if (t >= t_end) return 0.0;
        double rest = 0.5 * (t_end - t);
        if (dt >= rest) { dt = rest; *clipped = 1; }
    }
    return dt;
}

int orc_step(const orc_grid* g, double* const f[8], double* t, int* phase, double t_end,
             double* dt_out)
{
    int st = 0, clipped = 0;
    double dt = orc_dt(g, f, *t, t_end, &clipped, &st);
    if (dt_out) *dt_out = dt;
    if (dt <= 0.0) return st;
    st |= orc_step_dt(g, f, *phase, dt);
#if ORC_MUTANT == 12
    *t += dt;                                 /* mistake: a step advances 2 dt */
#else
    *t = clipped ? t_end : *t + 2.0 * dt;
#endif
    *phase = (*phase + 1) % 3;
    return st;
}

int orc_run(const orc_grid* g, double* const f[8], double* t, int* phase, int nsteps,
            double t_end, int* steps_done)
{
    int st = 0, k = 0;
    for (; k < nsteps; ++k) {
        double dt = 0.0;
        st |= orc_step(g, f, t, phase, t_end, &dt);
        if (dt <= 0.0) break;
    }
    if (steps_done) *steps_done = k;
    return st;
}

/* ------------------------------------------------------------------------------------ */
/* Diagnostics used by the pins.                                                           */
/* ------------------------------------------------------------------------------------ */

/* discrete divergence of the face field, summed over the faces of each cell */
double orc_divb_max(const orc_grid* g, double* const f[8])
{
    double m = 0.0;
    for (int x = 0; x < g->n[0]; ++x)
        for (int y = 0; y < g->n[1]; ++y)
            for (int z = 0; z < g->n[2]; ++z) {
                int c[3] = {x, y, z};
                long i0 = flat(g, c);
                double d = 0.0;
                for (int a = 0; a < 3; ++a) {
                    int cn[3] = {x, y, z};
                    cn[a] = imap(c[a] + 1, g->n[a], g->bc[a]);
                    d += f[5 + a][flat(g, cn)] - f[5 + a][i0];
                }
                d = fabs(d) / g->h;
                if (d > m) m = d;
            }
    return m;
}
