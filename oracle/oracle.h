/*
 * Plain FP64 CPU oracle for the unsplit piecewise-linear CTU step of the compressible solver
 * (paper §3.2 "Compressible hydrodynamics", Eqs. 8-13, with the CTU construction of §3.1, Eqs. 3-6).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no code, header, table or constant with the CUDA library; the two are
 * compared element by element on identical seeded inputs.
 *
 * Layout of a state array: U[k][j][i], k in {rho, rho*u, rho*v, rho*E}, j the row (y), i the column (x,
 * fastest), with NX = nx + 2 ng columns and NY = ny + 2 ng rows, contiguous.  Interior cells are
 * i in [ng, ng+nx), j in [ng, ng+ny).
 *
 * Every function is a straight transcription of the method's steps in the paper's order, one plain
 * loop per stage, with no blocking or fusion.  Status codes: 0 ok, 1 invalid arguments, 2 out of memory.
 */
#ifndef ORACLE_HYDRO_H
#define ORACLE_HYDRO_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, ng;
  double xmin, xmax, ymin, ymax;
  double gamma, cfl;
  int bc_xlo, bc_xhi, bc_ylo, bc_yhi; /* 0 outflow (zero gradient), 1 periodic, 2 reflecting,
                                          3 hydrostatic (y sides only) */
  int limiter;                         /* 0 piecewise constant, 1 MC, 2 fourth-order MC */
  int use_flattening;                  /* 0/1 */
  double cvisc;                        /* artificial-viscosity coefficient (0 disables) */
  int riemann_maxiter;
  double riemann_tol;
  double small_dens, small_pres;       /* floors applied to working copies only */
  double grav;                         /* constant gravitational acceleration along y (0: none) */
  int riemann_solver;                  /* 0 two-shock iteration, 1 HLLC */
  int reconstruction;                  /* 0 piecewise linear (limiter applies), 1 piecewise parabolic */
} oracle_params;

typedef struct {
  long long riemann_solves;     /* number of two-shock solves performed */
  long long riemann_iters;      /* total Newton iterations over all solves */
  long long riemann_nonconv;    /* solves that hit riemann_maxiter without meeting the tolerance */
  int riemann_maxiters_seen;
} oracle_stats;

/* ---- whole-grid driver calls (the solver's initialize/timestep/evolve sequence, paper §2) ---- */
int oracle_fill_ghost(const oracle_params* p, double* U);
int oracle_cfl_dt(const oracle_params* p, const double* U, double* dt_out);
int oracle_step(const oracle_params* p, double* U, double dt, oracle_stats* st);
int oracle_conserved_totals(const oracle_params* p, const double* U, double out[4]);
/* Dimensionally split step (§3.1): a one-dimensional sweep along first_dir (0: x, 1: y), a ghost fill of
 * the intermediate state, then a sweep along the other direction, each with the full dt.  The caller
 * alternates first_dir from step to step.  U must be ghost-filled on entry.  Gravity acts in the y sweep. */
int oracle_step_split(const oracle_params* p, double* U, double dt, int first_dir, oracle_stats* st);

/* ---- per-cell / per-face stages, exported so tests can pin each one on its own ---- */
void oracle_cons_to_prim(const oracle_params* p, const double U[4], double q[4]);
void oracle_prim_to_cons(const oracle_params* p, const double q[4], double U[4]);
double oracle_slope(int limiter, double qm2, double qm1, double q0, double qp1, double qp2);
double oracle_flatten_chi(double pm2, double pm1, double pp1, double pp2, double um1, double up1, double small_pres);
/* flattening coefficient of every cell from the primitives q [4][NY][NX] (rho, u, v, p planes) into
 * xi [NY][NX]: xi = min over x and y of min(chi_i, chi_{i-s}), s = sign(p_{i+1} - p_{i-1}); 0 ok, 2 no memory */
int oracle_flatten_xi(const oracle_params* p, const double* q, double* xi);
void oracle_trace(const oracle_params* p, double sigma, const double q[4], const double dq[4], double qL[4],
                  double qR[4]);
/* PPM: edge values (aL, aR) of the middle cell of a[0..4] after the monotonicity constraints and the
 * flattening blend xi; tracing of the parabolic profiles (aL, aR, and the cell average q) of the four
 * face-frame variables. */
void oracle_ppm_edges(const double a[5], double xi, double edges[2]);
void oracle_trace_ppm(const oracle_params* p, double sigma, const double q[4], const double aL[4], const double aR[4],
                      double qL[4], double qR[4]);
/* two-shock Riemann problem in the face frame: q = (rho, u_normal, u_transverse, p).
 * guess <= 0 selects the acoustic (linearised) initial guess.  Outputs the face state and the flux
 * (mass, normal momentum, transverse momentum, energy), the converged p* and u*, and the iteration count. */
int oracle_riemann(const oracle_params* p, const double qL[4], const double qR[4], double guess, double face[4],
                   double flux[4], double* pstar, double* ustar, int* iters);
void oracle_euler_flux(const oracle_params* p, const double q[4], double F[4]);
/* HLLC flux in the face frame (Toro 1997): oracle_hllc bounds the outer waves by the sound speeds of both
 * sides (Davis) and returns (S_L, S*, S_R) in speeds when not NULL; oracle_hllc_core takes S_L and S_R as
 * given and returns S* in *sstar when not NULL. */
void oracle_hllc(const oracle_params* p, const double qL[4], const double qR[4], double flux[4], double speeds[3]);
void oracle_hllc_core(const oracle_params* p, const double qL[4], const double qR[4], double SL, double SR,
                      double flux[4], double* sstar);

int oracle_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
