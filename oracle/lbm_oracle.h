/*
 * FP64 CPU oracle for the iD3Q14 / iD3Q18 incompressible MRT lattice
 * Boltzmann models (arXiv:1503.03337).  TEST INFRASTRUCTURE ONLY: nothing in
 * the CUDA library includes, links or calls this.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORACLE_PERIODIC = 0,
  ORACLE_WALL = 1,
  ORACLE_MOVING_WALL = 2,
  ORACLE_SYMMETRY = 3,
  /* Non-equilibrium extrapolation boundaries (Sec. 4, after Guo, Zheng and
   * Shi): the outermost node layer lies on the boundary.  After each step
   * every boundary node takes f = f_eq(p_b, u_b) + f(x_f) - f_eq(p_f, u_f),
   * x_f its inward neighbour, (p_f, u_f) the macroscopic values there. */
  ORACLE_NEQ_VELOCITY = 4, /* u_b = u_wall of the face, p_b = p_f        */
  ORACLE_NEQ_PRESSURE = 5  /* p_b = the face's pressure, u_b = u_f       */
};

typedef struct {
  int Q;              /* 14, 18 or 26 */
  int nx, ny, nz;     /* fluid nodes per axis */
  int face[6];        /* x-, x+, y-, y+, z-, z+ : ORACLE_* kinds */
  double u_wall[6][3];/* wall velocity of each MOVING_WALL face */
  /* Edge profile of a moving face (the corner velocities of Sec. 4.3): if
   * edge_axis[f] = k + 1, the wall velocity of face f seen from the first
   * (last) node column along axis k is u_wall[f] * edge_scale[f][0] ([1]);
   * a one-node axis takes [0].  0 = uniform. */
  int edge_axis[6];
  double edge_scale[6][2];
  /* Solid nodes (general geometry): NULL, or nx*ny*nz bytes, x fastest,
   * nonzero = solid.  A fluid node whose pull source is a solid node
   * bounces the population back as from a wall at rest halfway between
   * the two nodes; solid nodes hold no flow (their populations, velocity
   * and pressure are reported as zero). */
  const unsigned char *solid;
} oracle_grid;

typedef struct {
  double sc, se, sq, snu, spi, st; /* relaxation rates (spi unused for Q14) */
} oracle_rates;

typedef struct {
  oracle_rates rates;
  double force[3]; /* body force amplitude (lattice units) */
  double period;   /* > 0: F(t_n) = force cos(2 pi n / period); else constant */
  /* pressure of each ORACLE_NEQ_PRESSURE face at step n:
   * p_face[f] + p_amp[f] cos(2 pi n / p_period) (p_period > 0), else p_face[f] */
  double p_face[6];
  double p_amp[6];
  double p_period;
} oracle_params;

int oracle_velocities(int Q, int *c_out);           /* Q*3 ints */
int oracle_weights(int Q, double *w_out, double *w0_out);
int oracle_transform(int Q, double *T_out);         /* Q*Q, row-major */
int oracle_moment_equilibrium(int Q, double p, const double *u, double *meq);
int oracle_pressure(int Q, double P, const double *u, double *p);
int oracle_feq(int Q, double p, const double *u, double *feq);
int oracle_collide(int Q, const oracle_rates *r, const double *f,
                   const double *F, double *fpost);
int oracle_init_equilibrium(const oracle_grid *g, const double *u,
                            const double *p, double *f);
int oracle_step(const oracle_grid *g, const oracle_params *prm, int64_t n,
                const double *f_in, double *f_out, int nthreads);
int oracle_run(const oracle_grid *g, const oracle_params *prm, int64_t n0,
               int64_t nsteps, double *f, int nthreads);
int oracle_macroscopic(const oracle_grid *g, const oracle_params *prm,
                       int64_t n, const double *f, double *u, double *p);

#ifdef __cplusplus
}
#endif
#endif
