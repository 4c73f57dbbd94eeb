/*
 * oracle.h -- CPU oracle for the entropy-stable DG Euler solver with buoyancy
 * (Waterhouse, Waruszewski, Wilcox, Warburton, Giraldo: "GPU Performance of an
 * Entropy-Stable Discontinuous Galerkin Euler Solver with Non-Conservative
 * Terms").
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, single-threaded, deliberately slow
 * implementation of the semi-discrete right-hand side of Eq. (nm:semi) and of
 * the low-storage RK4 time stepping around it.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code with the CUDA library: not its kernels, headers, tables or helpers.
 *
 * The same source is compiled twice: with REAL = double (liboracle.so) and
 * REAL = long double (liboracle_ld.so).  The interface is always double; the
 * long-double build measures the double build's own rounding floor.
 *
 * Layouts (all row-major, element-major):
 *   state      q[e][v][n]       v = 0..4 : rho, rho u, rho v, rho w, E
 *   node       n = i + Nq*(j + Nq*k), (i,j,k) along reference (xi, eta, zeta)
 *   element    e = ex + Kx*(ey + Ky*ez)
 *   coords     x[e][c][n]       c = physical component
 *   metric     Ja[e][d][c][n]   d = reference direction, c = physical component
 *   Jacobian   J[e][n]
 */
#ifndef ES_DG_ORACLE_H
#define ES_DG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int kx, ky, kz;       /* elements per direction */
  double lo[3], hi[3];  /* box extents */
  int periodic[3];      /* 1 = periodic, 0 = reflecting wall */
  double warp;          /* warp amplitude as a fraction of the box edge; 0 = none */
} or_mesh;

typedef struct {
  double gamma, g, R, p0;  /* gas and gravity constants */
  double f0, beta, y0;     /* Coriolis parameter f = f0 + beta (y - y0) about z */
  int dissipation;         /* 1 = matrix dissipation at interfaces, 0 = EC only */
} or_phys;

typedef struct or_ctx or_ctx;

/* LGL nodes, weights and derivative matrix D[i][l]; Dt[i][l] = 2D - W^-1 B. */
int or_lgl(int N, double* xi, double* w, double* D, double* Dt);

or_ctx* or_create(const or_mesh* mesh, int N, const or_phys* phys);
void    or_free(or_ctx* c);
int     or_nelem(const or_ctx* c);
int     or_geometry(const or_ctx* c, double* x, double* J, double* Ja);

/* Semi-discrete right-hand side, Eq. (nm:semi); parts returns volume, surface
 * and source contributions separately (each may be NULL). */
int or_rhs(const or_ctx* c, const double* q, double* rhs);
int or_rhs_parts(const or_ctx* c, const double* q, double* vol, double* surf, double* src);
int or_rhs_scale(const or_ctx* c, const double* q, double* out);

/* Carpenter-Kennedy five-stage fourth-order 2N-storage RK. */
void or_lsrk_coeffs(double* A, double* B, double* c);
int  or_lsrk_steps(const or_ctx* c, double* q, double dt, int nsteps);

/* Initial states. */
int or_init_bubble(const or_ctx* c, double theta0, double amp, const double* centre,
                   double radius, double* q);
/* profile 0 = cosine bubble, Eq. (smooth-rb-ic); 1 = step bubble, Eq. (sharp-rb-ic) */
int or_init_bubble_profile(const or_ctx* c, double theta0, double amp, const double* centre,
                           double radius, int profile, double* q);
int or_init_isothermal(const or_ctx* c, double T, double rho_surface, double* q);
int or_init_channel(const or_ctx* c, double* q);

/* Global diagnostics: mass, total energy and entropy integrals; entropy rate. */
int    or_integrals(const or_ctx* c, const double* q, double* out3);
double or_entropy_rate(const or_ctx* c, const double* q, const double* rhs);
double or_cfl_dt(const or_ctx* c, const double* q, double C);

/* Pointwise building blocks (exported for the pin tests). */
double or_logmean(double a, double b);
void   or_entropy_vars(const double* q, double phi, double gamma, double* v);
void   or_ec_flux(const double* qa, double phia, const double* qb, double phib,
                  const double* n, double gamma, double* F, double* G);
void   or_es_flux(const double* qm, const double* qp, double phi, const double* nhat,
                  double gamma, int dissipation, double* Fstar);
void   or_dissipation_matrix(const double* qm, const double* qp, double phi,
                             const double* nhat, double gamma, double* Dmat);
void   or_eigensystem(const double* qm, const double* qp, double phi, const double* nhat,
                      double gamma, double* R, double* lam, double* T);

#ifdef __cplusplus
}
#endif
#endif
