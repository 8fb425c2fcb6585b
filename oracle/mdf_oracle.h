/*
 * FP64 CPU oracle of the MDF-LBM (arXiv 2108.08591).  TEST INFRASTRUCTURE
 * ONLY: used by the test-suite, the smoke check and the benchmark's CPU
 * baseline; never by the product library.  See mdf_oracle.c for the
 * equations each function follows.
 */
#ifndef MDF_ORACLE_H
#define MDF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int d;             /* spatial dimension, 2 or 3 */
    int q;             /* 5 (D2Q5) or 7 (D3Q7) */
    int with_rho;      /* 1: carry the alpha = 0 continuity set */
    int n[3];          /* nodes per axis; n[2] = 1 in 2D */
    int wall[3];       /* 1: halfway walls at both ends of the axis, 0: periodic */
    int lid;           /* 1: the + face of the last axis moves with lid_u */
    double lid_u[3];   /* lid velocity (physical units) */
    double dx, dt;     /* lattice spacing and time step */
    double s0, s1, s2; /* relaxation rates of S_d (Eq. 4-3) */
    double rho0;       /* constant density, ubar_0 */
    const double *force; /* nullable [d][N] body force at the nodes */
    int scheme;        /* forcing: 0 = Eq. 3-21, 2 = Scheme II (Eq. 2-3c, 2-7a) */
} orc_problem;

int orc_lattice(int d, int q, double c, double *cv, double *w, double *cs2);
int orc_moment_basis(int d, int q, double c, double s0, double s1, double s2,
                     double *M, double *S);
int orc_collision_matrix(int d, int q, double c, double s0, double s1, double s2,
                         double *Lam);
int orc_init(const orc_problem *pb, const double *P, const double *u, double *f);
int orc_init_neq(const orc_problem *pb, const double *P, const double *u, const double *G,
                 double *f);
int orc_mask(const orc_problem *pb, unsigned char *mask);
int orc_step(const orc_problem *pb, const double *Lam, const double *f, double *fnew);
int orc_run(const orc_problem *pb, long nsteps, double *f);
int orc_macro(const orc_problem *pb, const double *f, double *P, double *u, double *rho);
int orc_derived(const orc_problem *pb, const double *f, double *G, double *div,
                double *S, double *sigma, double *omega);
int orc_sums(const orc_problem *pb, const double *f, double *sums);
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
