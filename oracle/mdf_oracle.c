/*
 * FP64 CPU oracle of the multiple-distribution-function lattice Boltzmann
 * method (MDF-LBM) with the MRT collision of Chai, Shi & Zhan (arXiv 2108.08591).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * It is written to be read against the paper, not to be fast:
 *   - the lattices are the paper's tables (D2Q5 and D3Q7, Sec. 2.2; also
 *     D2Q4 and D3Q6, which have no rest direction);
 *   - the collision matrix is assembled densely as Lambda = M^-1 S M
 *     (Eq. 4-1) with M^-1 obtained by Gauss-Jordan elimination, not by any
 *     orthogonality shortcut;
 *   - one time step applies, node by node and in the paper's order:
 *       Eq. 2-7  (zeroth moments),
 *       Eq. 3-15 (pressure from the first moments, R = 0),
 *       Eq. 2-4  (linear equilibrium),
 *       Eq. 3-21 (f* = f - Lambda (f - f^eq) + dt w_i Fbar_alpha, Eq. 2-6),
 *     and then streams f* to x + c_i dt (periodic wrap or anti-halfway
 *     bounce-back at walls, Sec. 4);
 *   - the derived fields follow Eq. 3-16 .. 3-19.
 * With scheme = 2 the forcing is Scheme II of Sec. 3.2 instead: the state
 * is fbar = f - dt F / 2, advanced by Eq. 2-3c
 *   fbar* = fbar - Lambda (fbar - f^eq) + dt (I - Lambda / 2) F,
 * with ubar_alpha = sum_i fbar + dt Fbar_alpha / 2 (Eq. 2-7a) and P from
 * Eq. 3-15 taken over fbar.
 * Everything is in physical units: c = dx/dt and the lattice speeds scale
 * with c, so the paper's experiments can be run as printed.  Lattice units
 * are the special case dx = dt = 1.
 *
 * Readings of points the paper leaves open (each is also listed with the
 * design notes of the repository):
 *   - D3Q7 transformation matrix (the paper gives M for D2Q5 only): rows
 *     1, c_x, c_y, c_z, 7|c|^2 - 6c^2, 2c_x^2 - c_y^2 - c_z^2, c_y^2 - c_z^2
 *     with S = diag(s0, s1, s1, s1, s2, s2, s2).
 *   - Anti-halfway bounce-back (cited, formula not printed): walls sit half
 *     way between nodes and, for a link from fluid node x along c_i that
 *     crosses a wall,  f_{-i}(x, t+dt) = -f*_i(x, t) + 2 w_i ubar_wall,
 *     with ubar_wall = rho0 for alpha = 0 and the wall velocity component
 *     for alpha >= 1 (the moving lid on the + face of the last axis).
 *   - For alpha = 0, ubar_0 in Eq. 2-4 is taken from Eq. 2-7 (sum of f_0).
 *   - Scheme II: initialisation by the equilibrium means f = f^eq(P, u), so
 *     the stored state is fbar = f^eq - dt F / 2 with the force at t = 0;
 *     the derived fields take f^ne = f - f^eq with f = fbar + dt F / 2.
 *
 * Population layout: f[a][i][node], node = x + nx*(y + ny*z); set index a
 * maps to alpha = a when the continuity set is carried (with_rho = 1) and to
 * alpha = a + 1 otherwise (the paper allows omitting alpha = 0, Sec. 3.2).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "mdf_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 7

/* ---------------------------------------------------------------------- */
/* Lattices, Sec. 2.2: D2Q5 (c_s^2 = c^2/3), D3Q7 (c_s^2 = c^2/4), and    */
/* the lattices without a rest direction, D2Q4 (c_s^2 = c^2/2) and D3Q6   */
/* (c_s^2 = c^2/3), in the paper's direction order.                       */
/* ---------------------------------------------------------------------- */
int orc_lattice(int d, int q, double c, double *cv, double *w, double *cs2)
{
    int i, b;
    for (i = 0; i < QMAX * 3; ++i) cv[i] = 0.0;
    if (d == 2 && q == 4) {
        /* c_1..c_4 = (1,0), (0,1), (-1,0), (0,-1) times c (index 0..3 here) */
        static const int e[4][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
        for (i = 0; i < 4; ++i) {
            for (b = 0; b < 2; ++b) cv[3 * i + b] = e[i][b] * c;
            w[i] = 0.25;
        }
        *cs2 = c * c / 2.0;
        return 0;
    }
    if (d == 3 && q == 6) {
        /* c_1..c_6 = +-x, +-y, +-z times c (index 0..5 here) */
        static const int e[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                                    {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
        for (i = 0; i < 6; ++i) {
            for (b = 0; b < 3; ++b) cv[3 * i + b] = e[i][b] * c;
            w[i] = 1.0 / 6.0;
        }
        *cs2 = c * c / 3.0;
        return 0;
    }
    if (d == 2 && q == 5) {
        /* c_0..c_4 = (0,0), (1,0), (0,1), (-1,0), (0,-1) times c */
        static const int e[5][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}};
        for (i = 0; i < 5; ++i)
            for (b = 0; b < 2; ++b) cv[3 * i + b] = e[i][b] * c;
        w[0] = 1.0 / 3.0;
        for (i = 1; i < 5; ++i) w[i] = 1.0 / 6.0;
        *cs2 = c * c / 3.0;
        return 0;
    }
    if (d == 3 && q == 7) {
        /* c_0 = 0, c_1,2 = +-x, c_3,4 = +-y, c_5,6 = +-z, times c */
        static const int e[7][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},
                                    {0, -1, 0}, {0, 0, 1},  {0, 0, -1}};
        for (i = 0; i < 7; ++i)
            for (b = 0; b < 3; ++b) cv[3 * i + b] = e[i][b] * c;
        w[0] = 1.0 / 4.0;
        for (i = 1; i < 7; ++i) w[i] = 1.0 / 8.0;
        *cs2 = c * c / 4.0;
        return 0;
    }
    return -1;
}

/* Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix. */
static int invert(int n, const double *A, double *Ainv)
{
    double a[QMAX][2 * QMAX];
    int r, k, j, piv;
    for (r = 0; r < n; ++r)
        for (j = 0; j < 2 * n; ++j)
            a[r][j] = j < n ? A[r * n + j] : (j - n == r ? 1.0 : 0.0);
    for (k = 0; k < n; ++k) {
        double best = 0.0, p;
        piv = -1;
        for (r = k; r < n; ++r)
            if (fabs(a[r][k]) > best) { best = fabs(a[r][k]); piv = r; }
        if (piv < 0 || best == 0.0) return -1;
        if (piv != k)
            for (j = 0; j < 2 * n; ++j) { double t = a[k][j]; a[k][j] = a[piv][j]; a[piv][j] = t; }
        p = a[k][k];
        for (j = 0; j < 2 * n; ++j) a[k][j] /= p;
        for (r = 0; r < n; ++r) {
            double m;
            if (r == k) continue;
            m = a[r][k];
            if (m != 0.0)
                for (j = 0; j < 2 * n; ++j) a[r][j] -= m * a[k][j];
        }
    }
    for (r = 0; r < n; ++r)
        for (j = 0; j < n; ++j) Ainv[r * n + j] = a[r][n + j];
    return 0;
}

/* Transformation matrix M (q x q, row-major) and relaxation diagonal S.
 * D2Q5: Eq. 4-2 and Eq. 4-3.  D3Q7: the orthogonal analogue read above.
 * D2Q4 and D3Q6 (no M printed): the conserved row, the d first moments and
 * the traceless second moments of the same analogue (|c|^2 = c^2 is the
 * conserved row there), relaxed with s0, s1 and s2:
 *   D2Q4: 1, c_x, c_y, c_x^2 - c_y^2;
 *   D3Q6: 1, c_x, c_y, c_z, 2 c_x^2 - c_y^2 - c_z^2, c_y^2 - c_z^2. */
int orc_moment_basis(int d, int q, double c, double s0, double s1, double s2,
                     double *M, double *S)
{
    double cv[QMAX * 3], w[QMAX], cs2;
    int i;
    if (orc_lattice(d, q, c, cv, w, &cs2)) return -1;
    if (q == 4) {
        for (i = 0; i < 4; ++i) {
            double cx = cv[3 * i], cy = cv[3 * i + 1];
            M[0 * 4 + i] = 1.0;
            M[1 * 4 + i] = cx;
            M[2 * 4 + i] = cy;
            M[3 * 4 + i] = cx * cx - cy * cy;
        }
        S[0] = s0; S[1] = s1; S[2] = s1; S[3] = s2;
        return 0;
    }
    if (q == 6) {
        for (i = 0; i < 6; ++i) {
            double cx = cv[3 * i], cy = cv[3 * i + 1], cz = cv[3 * i + 2];
            M[0 * 6 + i] = 1.0;
            M[1 * 6 + i] = cx;
            M[2 * 6 + i] = cy;
            M[3 * 6 + i] = cz;
            M[4 * 6 + i] = 2.0 * cx * cx - cy * cy - cz * cz;
            M[5 * 6 + i] = cy * cy - cz * cz;
        }
        S[0] = s0; S[1] = s1; S[2] = s1; S[3] = s1; S[4] = s2; S[5] = s2;
        return 0;
    }
    if (d == 2) {
        for (i = 0; i < 5; ++i) {
            double cx = cv[3 * i], cy = cv[3 * i + 1];
            M[0 * 5 + i] = 1.0;
            M[1 * 5 + i] = cx;
            M[2 * 5 + i] = cy;
            M[3 * 5 + i] = cx * cx - cy * cy;              /* (0, c^2, -c^2, c^2, -c^2) */
            M[4 * 5 + i] = i == 0 ? -4.0 * c * c : c * c;  /* (-4c^2, c^2, c^2, c^2, c^2) */
        }
        S[0] = s0; S[1] = s1; S[2] = s1; S[3] = s2; S[4] = s2;
        return 0;
    }
    for (i = 0; i < 7; ++i) {
        double cx = cv[3 * i], cy = cv[3 * i + 1], cz = cv[3 * i + 2];
        double c2 = cx * cx + cy * cy + cz * cz;
        M[0 * 7 + i] = 1.0;
        M[1 * 7 + i] = cx;
        M[2 * 7 + i] = cy;
        M[3 * 7 + i] = cz;
        M[4 * 7 + i] = 7.0 * c2 - 6.0 * c * c;
        M[5 * 7 + i] = 2.0 * cx * cx - cy * cy - cz * cz;
        M[6 * 7 + i] = cy * cy - cz * cz;
    }
    S[0] = s0; S[1] = s1; S[2] = s1; S[3] = s1; S[4] = s2; S[5] = s2; S[6] = s2;
    return 0;
}

/* Eq. 4-1: Lambda = M^-1 S_d M, dense q x q. */
int orc_collision_matrix(int d, int q, double c, double s0, double s1, double s2,
                         double *Lam)
{
    double M[QMAX * QMAX], Minv[QMAX * QMAX], S[QMAX];
    int i, j, k;
    if (orc_moment_basis(d, q, c, s0, s1, s2, M, S)) return -1;
    if (invert(q, M, Minv)) return -1;
    for (i = 0; i < q; ++i)
        for (j = 0; j < q; ++j) {
            double acc = 0.0;
            for (k = 0; k < q; ++k) acc += Minv[i * q + k] * S[k] * M[k * q + j];
            Lam[i * q + j] = acc;
        }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Problem description helpers                                            */
/* ---------------------------------------------------------------------- */
static long nnodes(const orc_problem *pb) { return (long)pb->n[0] * pb->n[1] * pb->n[2]; }
static int nsets(const orc_problem *pb) { return pb->with_rho ? pb->d + 1 : pb->d; }
static int alpha_of(const orc_problem *pb, int a) { return pb->with_rho ? a : a + 1; }

static int check(const orc_problem *pb)
{
    int b;
    if (!((pb->d == 2 && (pb->q == 5 || pb->q == 4)) || (pb->d == 3 && (pb->q == 7 || pb->q == 6))))
        return -1;
    for (b = 0; b < 3; ++b)
        if (pb->n[b] < 1) return -1;
    if (pb->d == 2 && pb->n[2] != 1) return -1;
    if (!(pb->dx > 0.0) || !(pb->dt > 0.0)) return -1;
    if (pb->scheme != 0 && pb->scheme != 2) return -1;
    return 0;
}

/* Fbar_alpha at a node (alpha >= 1; zero without a force or for alpha = 0). */
static double force_at(const orc_problem *pb, int alpha, long node, long N)
{
    if (alpha < 1 || !pb->force) return 0.0;
    return pb->force[(long)(alpha - 1) * N + node];
}

/* dt F_{i,alpha} / 2 = dt w_i Fbar_alpha / 2: the change of variable of
 * Scheme II (fbar = f - dt F / 2); zero for the Eq. 3-21 forcing. */
static double half_source(const orc_problem *pb, const double *w, int i, int alpha,
                          long node, long N)
{
    if (pb->scheme != 2) return 0.0;
    return 0.5 * pb->dt * w[i] * force_at(pb, alpha, node, N);
}

static int opposite(const double *cv, int q, int i)
{
    int j;
    for (j = 0; j < q; ++j)
        if (cv[3 * j] == -cv[3 * i] && cv[3 * j + 1] == -cv[3 * i + 1] &&
            cv[3 * j + 2] == -cv[3 * i + 2])
            return j;
    return -1;
}

/* Lattice direction of c_i as integers (c_i / c). */
static void unit_dir(const double *cv, double c, int i, int e[3])
{
    int b;
    for (b = 0; b < 3; ++b) e[b] = (int)lround(cv[3 * i + b] / c);
}

/* Eq. 2-4: equilibrium of set alpha at one node. */
static void equilibrium(int q, int d, int alpha, const double *cv, const double *w,
                        double cs2, double ubar, const double *u, double P,
                        double *feq)
{
    int i, b;
    for (i = 0; i < q; ++i) {
        double flux = 0.0;
        for (b = 0; b < d; ++b) {
            double Fb = ubar * u[b] + ((alpha >= 1 && b == alpha - 1) ? P : 0.0);
            flux += cv[3 * i + b] * Fb;
        }
        feq[i] = w[i] * (ubar + flux / cs2);
    }
}

/* Eq. 2-7 and Eq. 3-15 at one node: ubar_a for every set, u, P.  Under
 * Scheme II f holds fbar: ubar_a = sum_i fbar + dt Fbar_a / 2 (Eq. 2-7a) and
 * the first moments in P are those of fbar. */
static void macroscopic(const orc_problem *pb, const double *cv, const double *f,
                        long node, long N, double *ubar, double *u, double *P)
{
    int q = pb->q, d = pb->d, ns = nsets(pb), a, i, b;
    double first = 0.0, usq = 0.0;
    for (a = 0; a < ns; ++a) {
        double s = 0.0;
        for (i = 0; i < q; ++i) s += f[((long)a * q + i) * N + node];
        if (pb->scheme == 2) s += 0.5 * pb->dt * force_at(pb, alpha_of(pb, a), node, N);
        ubar[a] = s;
    }
    for (b = 0; b < d; ++b) {
        int a_of = pb->with_rho ? b + 1 : b; /* set index of alpha = b + 1 */
        u[b] = ubar[a_of];
        usq += u[b] * u[b];
        /* sum_i c_{i,alpha} f_{i,alpha} with alpha = b + 1 */
        for (i = 0; i < q; ++i) first += cv[3 * i + b] * f[((long)a_of * q + i) * N + node];
    }
    /* R = 0 in every workload here, so the (dt/s1) c_s^2 R term vanishes. */
    *P = (first - usq) / d;
}

/* ---------------------------------------------------------------------- */
/* Initialisation: f = f^eq(P, u) (Sec. 4, "initialization ... by their    */
/* equilibrium distribution functions"), optionally plus the first-order  */
/* non-equilibrium part of a given velocity gradient.                     */
/* ---------------------------------------------------------------------- */

/* First-order non-equilibrium part of set alpha >= 1 for the velocity
 * gradient G[a][b] = d u_a / d x_b at one node.  The first moment of
 * f^ne relaxes with s1 (Eq. 4-3), and D_i f^eq_{i,alpha} carries
 * w_i (c_i . grad) ubar_alpha at first order, which has first moments only,
 * so Lambda^-1 acts on it as 1/s1:
 *   f^ne_{i,alpha} = -(dt / s1) w_i sum_b c_{i,b} (G[alpha-1][b] - delta tr(G) / d).
 * Its first moment is -(c_s^2 dt / s1) times the traceless gradient: the
 * inverse of Eq. 3-16.  The trace is removed because Eq. 3-15 reads the
 * trace of the first moments as pressure; the seeded P is kept.  The
 * alpha = 0 set gets none (its first-order part is O(u grad u)). */
static void neq_part(const orc_problem *pb, const double *cv, const double *w, int alpha,
                     const double *G, long node, long N, double *fne)
{
    int d = pb->d, i, b;
    double tr = 0.0;
    for (i = 0; i < pb->q; ++i) fne[i] = 0.0;
    if (alpha < 1 || !G) return;
    for (b = 0; b < d; ++b) tr += G[((long)b * d + b) * N + node];
    for (i = 0; i < pb->q; ++i) {
        double s = 0.0;
        for (b = 0; b < d; ++b) {
            double g = G[((long)(alpha - 1) * d + b) * N + node];
            if (b == alpha - 1) g -= tr / d;
            s += cv[3 * i + b] * g;
        }
        fne[i] = -(pb->dt / pb->s1) * w[i] * s;
    }
}

int orc_init_neq(const orc_problem *pb, const double *P, const double *u, const double *G,
                 double *f)
{
    double cv[QMAX * 3], w[QMAX], cs2, c;
    long N, n;
    int ns, a;
    if (check(pb)) return -1;
    c = pb->dx / pb->dt;
    orc_lattice(pb->d, pb->q, c, cv, w, &cs2);
    N = nnodes(pb);
    ns = nsets(pb);
    for (n = 0; n < N; ++n) {
        double un[3], feq[QMAX], fne[QMAX];
        int b, i;
        for (b = 0; b < pb->d; ++b) un[b] = u[(long)b * N + n];
        for (a = 0; a < ns; ++a) {
            int alpha = alpha_of(pb, a);
            double ubar = alpha == 0 ? pb->rho0 : un[alpha - 1];
            equilibrium(pb->q, pb->d, alpha, cv, w, cs2, ubar, un, P[n], feq);
            neq_part(pb, cv, w, alpha, G, n, N, fne);
            /* Scheme II stores fbar = f - dt F / 2 */
            for (i = 0; i < pb->q; ++i)
                f[((long)a * pb->q + i) * N + n] =
                    feq[i] + fne[i] - half_source(pb, w, i, alpha, n, N);
        }
    }
    return 0;
}

int orc_init(const orc_problem *pb, const double *P, const double *u, double *f)
{
    return orc_init_neq(pb, P, u, NULL, f);
}

/* ---------------------------------------------------------------------- */
/* Boundary geometry: bit i of mask[node] is set when the link from node  */
/* along c_i crosses a wall; bit 7 is set when one of them crosses the    */
/* moving lid (the + face of the last axis).                              */
/* ---------------------------------------------------------------------- */
static int crosses(const orc_problem *pb, const int x[3], const int e[3], int *lid)
{
    int b, hit = 0;
    *lid = 0;
    for (b = 0; b < pb->d; ++b) {
        int t = x[b] + e[b];
        if (pb->wall[b] && (t < 0 || t >= pb->n[b])) {
            hit = 1;
            if (pb->lid && b == pb->d - 1 && t >= pb->n[b]) *lid = 1;
        }
    }
    return hit;
}

int orc_mask(const orc_problem *pb, unsigned char *mask)
{
    double cv[QMAX * 3], w[QMAX], cs2, c;
    long N, n;
    if (check(pb)) return -1;
    c = pb->dx / pb->dt;
    orc_lattice(pb->d, pb->q, c, cv, w, &cs2);
    N = nnodes(pb);
    for (n = 0; n < N; ++n) {
        int x[3], i, e[3], lid;
        unsigned char m = 0;
        x[0] = (int)(n % pb->n[0]);
        x[1] = (int)((n / pb->n[0]) % pb->n[1]);
        x[2] = (int)(n / ((long)pb->n[0] * pb->n[1]));
        for (i = 0; i < pb->q; ++i) {
            unit_dir(cv, c, i, e);
            if (crosses(pb, x, e, &lid)) {
                m |= (unsigned char)(1u << i);
                if (lid) m |= 0x80u;
            }
        }
        mask[n] = m;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* One time step of Eq. 3-21 (Eq. 2-3c under Scheme II) and streaming.   */
/* f holds f(x, t) (post-stream); fnew receives f(x, t + dt).             */
/* ---------------------------------------------------------------------- */
int orc_step(const orc_problem *pb, const double *Lam, const double *f, double *fnew)
{
    double cv[QMAX * 3], w[QMAX], cs2, c;
    long N;
    int ns, q, d;
    if (check(pb)) return -1;
    c = pb->dx / pb->dt;
    orc_lattice(pb->d, pb->q, c, cv, w, &cs2);
    N = nnodes(pb);
    ns = nsets(pb);
    q = pb->q;
    d = pb->d;

#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double ubar[4], u[3], P, feq[QMAX], fstar[QMAX];
        int x[3], a, i, k, b;
        x[0] = (int)(n % pb->n[0]);
        x[1] = (int)((n / pb->n[0]) % pb->n[1]);
        x[2] = (int)(n / ((long)pb->n[0] * pb->n[1]));

        macroscopic(pb, cv, f, n, N, ubar, u, &P); /* Eq. 2-7, Eq. 3-15 */

        for (a = 0; a < ns; ++a) {
            int alpha = alpha_of(pb, a);
            const double *fa = f + (long)a * q * N;
            /* Eq. 2-6: F_i = w_i Fbar_alpha; Fbar_0 = R = 0 */
            const double Fbar = force_at(pb, alpha, n, N);
            equilibrium(q, d, alpha, cv, w, cs2, ubar[a], u, P, feq); /* Eq. 2-4 */
            for (i = 0; i < q; ++i) {
                double coll = 0.0, src = 0.0;
                for (k = 0; k < q; ++k) coll += Lam[i * q + k] * (fa[k * N + n] - feq[k]);
                if (pb->scheme == 2) /* Eq. 2-3c: dt (delta_ik - Lambda_ik / 2) F_k */
                    for (k = 0; k < q; ++k)
                        src += ((k == i ? 1.0 : 0.0) - 0.5 * Lam[i * q + k]) * w[k] * Fbar;
                else                 /* Eq. 3-21: dt F_i */
                    src = w[i] * Fbar;
                fstar[i] = fa[i * N + n] - coll + pb->dt * src;
            }
            /* streaming to x + c_i dt, periodic or anti-halfway bounce-back */
            for (i = 0; i < q; ++i) {
                int e[3], lid, t[3];
                long m;
                unit_dir(cv, c, i, e);
                if (crosses(pb, x, e, &lid)) {
                    double uw = alpha == 0 ? pb->rho0 : (lid ? pb->lid_u[alpha - 1] : 0.0);
                    int io = opposite(cv, q, i);
                    fnew[((long)a * q + io) * N + n] = -fstar[i] + 2.0 * w[i] * uw;
                    continue;
                }
                for (b = 0; b < 3; ++b) {
                    t[b] = x[b] + e[b];
                    if (t[b] < 0) t[b] += pb->n[b];
                    if (t[b] >= pb->n[b]) t[b] -= pb->n[b];
                }
                m = t[0] + (long)pb->n[0] * (t[1] + (long)pb->n[1] * t[2]);
                fnew[((long)a * q + i) * N + m] = fstar[i];
            }
        }
    }
    return 0;
}

int orc_run(const orc_problem *pb, long nsteps, double *f)
{
    double Lam[QMAX * QMAX];
    double *g;
    long N, s, len;
    if (check(pb)) return -1;
    if (orc_collision_matrix(pb->d, pb->q, pb->dx / pb->dt, pb->s0, pb->s1, pb->s2, Lam))
        return -1;
    N = nnodes(pb);
    len = (long)nsets(pb) * pb->q * N;
    g = (double *)malloc(sizeof(double) * (size_t)len);
    if (!g) return -2;
    for (s = 0; s < nsteps; ++s) {
        orc_step(pb, Lam, f, g);
        memcpy(f, g, sizeof(double) * (size_t)len);
    }
    free(g);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Readouts                                                               */
/* ---------------------------------------------------------------------- */
int orc_macro(const orc_problem *pb, const double *f, double *P, double *u, double *rho)
{
    double cv[QMAX * 3], w[QMAX], cs2, c;
    long N, n;
    if (check(pb)) return -1;
    c = pb->dx / pb->dt;
    orc_lattice(pb->d, pb->q, c, cv, w, &cs2);
    N = nnodes(pb);
    for (n = 0; n < N; ++n) {
        double ubar[4], un[3], Pn;
        int b;
        macroscopic(pb, cv, f, n, N, ubar, un, &Pn);
        if (P) P[n] = Pn;
        if (u)
            for (b = 0; b < pb->d; ++b) u[(long)b * N + n] = un[b];
        if (rho && pb->with_rho) rho[n] = ubar[0];
    }
    return 0;
}

/*
 * Eq. 3-16 .. 3-19 from the first moments of f^ne = f - f^eq at the state
 * held in f.  Output layouts (each nullable):
 *   G[(a*d + b)*N + n]  = d u_a / d x_b      (Eq. 3-16, a, b = 0..d-1)
 *   div[n]                                     (Eq. 3-16a)
 *   S[k*N + n], sigma[k*N + n] over the upper triangle a <= b in row order
 *     2D: xx, xy, yy      3D: xx, xy, xz, yy, yz, zz    (Eq. 3-17, 3-17a)
 *   omega: 2D one component (du2/dx - du1/dy); 3D three (Eq. 3-18, 3-19)
 */
int orc_derived(const orc_problem *pb, const double *f, double *G, double *div,
                double *S, double *sigma, double *omega)
{
    double cv[QMAX * 3], w[QMAX], cs2, c, pref;
    long N, n;
    int d, q;
    if (check(pb)) return -1;
    c = pb->dx / pb->dt;
    orc_lattice(pb->d, pb->q, c, cv, w, &cs2);
    N = nnodes(pb);
    d = pb->d;
    q = pb->q;
    pref = -pb->s1 / (cs2 * pb->dt);
    for (n = 0; n < N; ++n) {
        double ubar[4], u[3], P, feq[QMAX], mne[3][3], grad[3][3];
        int a, b, i, k;
        macroscopic(pb, cv, f, n, N, ubar, u, &P);
        /* mne[a][b] = sum_i c_{i,b} f^ne_{i,alpha}, alpha = a + 1 */
        for (a = 0; a < d; ++a) {
            int set = pb->with_rho ? a + 1 : a;
            equilibrium(q, d, a + 1, cv, w, cs2, ubar[set], u, P, feq);
            for (b = 0; b < d; ++b) {
                double s = 0.0;
                for (i = 0; i < q; ++i) {
                    /* f = fbar + dt F / 2 under Scheme II */
                    double fi = f[((long)set * q + i) * N + n] + half_source(pb, w, i, a + 1, n, N);
                    s += cv[3 * i + b] * (fi - feq[i]);
                }
                mne[a][b] = s;
            }
        }
        for (a = 0; a < d; ++a)
            for (b = 0; b < d; ++b) grad[a][b] = pref * mne[a][b]; /* Eq. 3-16 */
        if (G)
            for (a = 0; a < d; ++a)
                for (b = 0; b < d; ++b) G[((long)a * d + b) * N + n] = grad[a][b];
        if (div) { /* Eq. 3-16a */
            double s = 0.0;
            for (a = 0; a < d; ++a) s += mne[a][a];
            div[n] = pref * s;
        }
        k = 0;
        for (a = 0; a < d; ++a)
            for (b = a; b < d; ++b, ++k) {
                double sym = mne[a][b] + mne[b][a];
                if (S) S[(long)k * N + n] = 0.5 * pref * sym;                        /* Eq. 3-17 */
                if (sigma) sigma[(long)k * N + n] = -pb->rho0 * (1.0 - 0.5 * pb->s1) * sym; /* Eq. 3-17a */
            }
        if (omega) {
            /* Eq. 3-18: Omega_ab = (pref/2)(mne[a][b] - mne[b][a]); Eq. 3-19:
             * Omega_ab = -1/2 eps_abg omega_g, so omega_g = -eps_abg Omega_ab
             * summed over the pair (a, b) and (b, a). */
            double Om[3][3];
            for (a = 0; a < d; ++a)
                for (b = 0; b < d; ++b) Om[a][b] = 0.5 * pref * (mne[a][b] - mne[b][a]);
            if (d == 2) {
                omega[n] = -2.0 * Om[0][1]; /* eps_{12 3} = 1 */
            } else {
                omega[0 * N + n] = -2.0 * Om[1][2];
                omega[1 * N + n] = -2.0 * Om[2][0];
                omega[2 * N + n] = -2.0 * Om[0][1];
            }
        }
    }
    return 0;
}

/* Sum over all nodes of ubar_a (Eq. 2-7; Eq. 2-7a under Scheme II) for
 * every carried set. */
int orc_sums(const orc_problem *pb, const double *f, double *sums)
{
    long N, n;
    int ns, a, i;
    if (check(pb)) return -1;
    N = nnodes(pb);
    ns = nsets(pb);
    for (a = 0; a < ns; ++a) {
        double s = 0.0;
        for (n = 0; n < N; ++n) {
            for (i = 0; i < pb->q; ++i) s += f[((long)a * pb->q + i) * N + n];
            if (pb->scheme == 2) s += 0.5 * pb->dt * force_at(pb, alpha_of(pb, a), n, N);
        }
        sums[a] = s;
    }
    return 0;
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
