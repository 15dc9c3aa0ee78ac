/*
 * FP64 CPU oracle for the iD3Q14 / iD3Q18 incompressible MRT lattice
 * Boltzmann models (Zhang, Shi & Wang, arXiv:1503.03337), and for the
 * iD3Q26 model that App. B's closing remark says the same construction
 * gives (built here by Sec. 3's recipe: moment monomials on the D3Q27 set
 * without c_0, Gram-Schmidt orthogonalised, m_eq = T f_eq).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header or
 * table with the CUDA library.
 *
 * Everything is double precision and is meant to be compiled with
 * -ffp-contract=off so that no multiply-add is fused behind the reader's back.
 *
 * The update follows the paper's order (Sec. 3, Eq. mrteqvT):
 *   1. P = sum f, j = sum c f                       (Eq. hgl)
 *   2. u = j + F/2, p from P and |u|^2               (Eq. hgl; Guo forcing)
 *   3. m = T f with the printed T                    (Eq. T14 / App. B;
 *                                                      iD3Q26: built T)
 *   4. m_eq from the printed closed forms            (Eq. meq / App. B;
 *                                                      iD3Q26: T f_eq)
 *   5. S_F = T Fbar, P row dropped                   (Guo forcing)
 *   6. m* = m - S (m - m_eq) + (I - S/2) S_F         (Eq. mrteqvT, diagonal S)
 *   7. f* = T^-1 m* with T^-1 = T' D^-1              (rows of T are orthogonal)
 *   8. pull streaming; a link whose source lies beyond a wall takes the
 *      cell's own reflected population plus 6 w (c . u_wall)
 *      (halfway and moving-wall bounce-back)
 *      A source that is a solid node of the grid's solid mask is a wall
 *      link at rest (halfway bounce-back off an arbitrary solid)
 *   9. non-equilibrium extrapolation (Sec. 4, the boundary scheme the paper
 *      always applies): every node on a face of kind ORACLE_NEQ_* takes
 *      f = f_eq(p_b, u_b) + [f(x_f) - f_eq(p_f, u_f)] from its inward
 *      neighbour x_f, with u_b given on velocity faces (p_b = p_f) and p_b
 *      given on pressure faces (u_b = u_f)
 *
 * Layout of every population array: f[a][z][y][x], a = 0..Q-1 holding the
 * paper's 1-based direction a+1, x fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "lbm_oracle.h"

/* ---- velocity sets ---------------------------------------------------- */

/* D3Q14 directions c_1..c_14 (Sec. 3, the velocity set of the iD3Q14 model) */
static const int C14[14][3] = {
    {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0}, {0, 0, 1},
    {0, 0, -1}, {1, 1, 1},   {-1, 1, 1}, {1, -1, 1}, {-1, -1, 1},
    {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};

/* D3Q18 directions c_1..c_18 (App. B, Eq. D3Q19) */
static const int C18[18][3] = {
    {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, 1, 0},  {1, -1, 0}, {-1, -1, 0}, {1, 0, 1},  {-1, 0, 1},
    {1, 0, -1}, {-1, 0, -1}, {0, 1, 1},  {0, -1, 1},  {0, 1, -1}, {0, -1, -1}};

/* D3Q26 directions: the D3Q27 set without c_0, ordered as the axes and face
 * diagonals of D3Q18 followed by the cube diagonals of D3Q14 */
static const int C26[26][3] = {
    {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},  {-1, 1, 0},  {1, -1, 0},  {-1, -1, 0}, {1, 0, 1},   {-1, 0, 1},
    {1, 0, -1}, {-1, 0, -1}, {0, 1, 1},   {0, -1, 1},  {0, 1, -1},  {0, -1, -1},
    {1, 1, 1},  {-1, 1, 1},  {1, -1, 1},  {-1, -1, 1}, {1, 1, -1},  {-1, 1, -1},
    {1, -1, -1}, {-1, -1, -1}};

/* ---- transformation matrices, as printed ------------------------------ */

/* Eq. T14 */
static const int T14[14][14] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -4, -4, -4, -4, -4, 3, 3, 3, 3, 3, 3, 3, 3},
    {1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
    {-4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
    {0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1},
    {0, 0, 0, 0, -4, 4, 1, 1, 1, 1, -1, -1, -1, -1},
    {2, 2, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1},
    {0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1},
    {0, 0, 0, 0, 0, 0, 1, -1, -1, 1, -1, 1, 1, -1}};

/* App. B, the 18x18 transformation matrix */
static const int T18[18][18] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-2, -2, -2, -2, -2, -2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {-4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, 0, -4, 4, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {2, 2, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {-4, -4, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, 0, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, -2, -2, 2, 2, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, -1, -1, 1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1}};

/* ---- model description ------------------------------------------------- */

typedef struct {
  int Q;
  const int (*c)[3];
  double T[26 * 26]; /* Q*Q, row-major */
  double w[26]; /* lattice weights of the directions actually stored */
  double w0;    /* weight of the discarded rest direction c_0 */
  double D[26]; /* D_k = sum_a T_ka^2 (row norms; T T' = diag(D)) */
} model;

/* The iD3Q26 moment polynomials, in row order: the 18 moments of the iD3Q18
 * basis (P, e, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww,
 * p_xy, p_yz, p_xz, t_x, t_y, t_z), then |c|^4, |c|^4 c_x, |c|^4 c_y,
 * |c|^4 c_z, |c|^2 c_x c_y, |c|^2 c_y c_z, |c|^2 c_x c_z and c_x c_y c_z:
 * the monomials of Sec. 3's recipe (Eq. transformation_Mbar) for the 26
 * velocities of D3Q27 without c_0.  c_x^2 c_y^2 c_z^2 is left out: on these
 * velocities (1 - c_x^2)(1 - c_y^2)(1 - c_z^2) = 0 makes it a combination of
 * the others, as the paper drops the kinetic-energy-square moment for Q14. */
static double poly26(int k, const int c[3]) {
  const double x = c[0], y = c[1], z = c[2];
  const double n2 = x * x + y * y + z * z;
  switch (k) {
    case 0: return 1.0;
    case 1: return n2;
    case 2: return x;
    case 3: return n2 * x;
    case 4: return y;
    case 5: return n2 * y;
    case 6: return z;
    case 7: return n2 * z;
    case 8: return 3.0 * x * x - n2;
    case 9: return n2 * (3.0 * x * x - n2);
    case 10: return y * y - z * z;
    case 11: return n2 * (y * y - z * z);
    case 12: return x * y;
    case 13: return y * z;
    case 14: return x * z;
    case 15: return x * (y * y - z * z);
    case 16: return y * (z * z - x * x);
    case 17: return z * (x * x - y * y);
    case 18: return n2 * n2;
    case 19: return n2 * n2 * x;
    case 20: return n2 * n2 * y;
    case 21: return n2 * n2 * z;
    case 22: return n2 * x * y;
    case 23: return n2 * y * z;
    case 24: return n2 * x * z;
    case 25: return x * y * z;
  }
  return 0.0;
}

static int model_init(int Q, model *m) {
  if (Q == 14) {
    m->Q = 14;
    m->c = C14;
    for (int k = 0; k < 14 * 14; ++k) m->T[k] = (double)(&T14[0][0])[k];
    /* The weights printed beside Eq. edf belong to D3Q19; the
     * Q14 equilibria of Eq. meq hold only with the D3Q15 weights
     * w0 = 2/9, 1/9 on the axes and 1/72 on the cube diagonals. */
    m->w0 = 2.0 / 9.0;
    for (int a = 0; a < 14; ++a) m->w[a] = (a < 6) ? 1.0 / 9.0 : 1.0 / 72.0;
  } else if (Q == 18) {
    m->Q = 18;
    m->c = C18;
    for (int k = 0; k < 18 * 18; ++k) m->T[k] = (double)(&T18[0][0])[k];
    /* App. B: w_1..6 = 1/18, w_7..18 = 1/36, so w0 = 1/3 */
    m->w0 = 1.0 / 3.0;
    for (int a = 0; a < 18; ++a) m->w[a] = (a < 6) ? 1.0 / 18.0 : 1.0 / 36.0;
  } else if (Q == 26) {
    /* iD3Q26 (App. B's closing remark): the D3Q27 weights 8/27, 2/27, 1/54,
     * 1/216 and the recipe of Sec. 3: the moment polynomials on the velocity
     * set, Gram-Schmidt orthogonalised in row order (Eq. transformation_Mbar) */
    m->Q = 26;
    m->c = C26;
    m->w0 = 8.0 / 27.0;
    for (int a = 0; a < 26; ++a)
      m->w[a] = a < 6 ? 2.0 / 27.0 : (a < 18 ? 1.0 / 54.0 : 1.0 / 216.0);
    for (int k = 0; k < 26; ++k) {
      double *row = &m->T[k * 26];
      for (int a = 0; a < 26; ++a) row[a] = poly26(k, C26[a]);
      for (int l = 0; l < k; ++l) {
        const double *prev = &m->T[l * 26];
        double num = 0.0, den = 0.0;
        for (int a = 0; a < 26; ++a) {
          num += row[a] * prev[a];
          den += prev[a] * prev[a];
        }
        for (int a = 0; a < 26; ++a) row[a] -= num / den * prev[a];
      }
      /* clear denominators, as the printed T14 and T18 are integer: the
       * smallest multiple of the row's smallest entry that makes every
       * entry an integer (the rows are rational with small denominators) */
      double small = 0.0;
      for (int a = 0; a < 26; ++a)
        if (fabs(row[a]) > 1e-9 && (small == 0.0 || fabs(row[a]) < small)) small = fabs(row[a]);
      int mult = 1;
      for (; mult <= 720; ++mult) {
        int ok = 1;
        for (int a = 0; a < 26 && ok; ++a) {
          const double v = row[a] * mult / small;
          ok = fabs(v - nearbyint(v)) < 1e-8;
        }
        if (ok) break;
      }
      if (mult > 720) return -1;
      for (int a = 0; a < 26; ++a) row[a] = nearbyint(row[a] * mult / small);
    }
  } else {
    return -1;
  }
  for (int k = 0; k < m->Q; ++k) {
    double s = 0.0;
    for (int a = 0; a < m->Q; ++a) {
      const double t = m->T[k * m->Q + a];
      s += t * t;
    }
    m->D[k] = s;
  }
  return 0;
}

static int opposite(const model *m, int a) {
  for (int b = 0; b < m->Q; ++b)
    if (m->c[b][0] == -m->c[a][0] && m->c[b][1] == -m->c[a][1] &&
        m->c[b][2] == -m->c[a][2])
      return b;
  return -1;
}

/* Diagonal of the collision matrix in moment order.
 * Q14: Eq. sD3Q15meaning, (sc,se,sc,sq,sc,sq,sc,sq,snu x5,st).
 * Q18: Eq. sD3Q19, (sc,se,sc,sq,sc,sq,sc,sq,snu,spi,snu,spi,snu,snu,snu,st x3). */
static void relaxation_diag(const model *m, const oracle_rates *r, double *s) {
  if (m->Q == 26) {
    /* the paper gives no rates for iD3Q26; the reading extends Eq. sD3Q19:
     * conserved s_c; e and |c|^4 s_e; the heat fluxes (q and the |c|^4 c
     * rows) s_q; the stress rows s_nu; the |c|^2-weighted stress rows s_pi;
     * the third-order rows t and c_x c_y c_z s_t */
    const double v[26] = {r->sc,  r->se,  r->sc,  r->sq,  r->sc,  r->sq,  r->sc,
                          r->sq,  r->snu, r->spi, r->snu, r->spi, r->snu, r->snu,
                          r->snu, r->st,  r->st,  r->st,  r->se,  r->sq,  r->sq,
                          r->sq,  r->spi, r->spi, r->spi, r->st};
    memcpy(s, v, sizeof v);
  } else if (m->Q == 14) {
    const double v[14] = {r->sc,  r->se,  r->sc,  r->sq,  r->sc,  r->sq,  r->sc,
                          r->sq,  r->snu, r->snu, r->snu, r->snu, r->snu, r->st};
    memcpy(s, v, sizeof v);
  } else {
    const double v[18] = {r->sc,  r->se,  r->sc,  r->sq,  r->sc, r->sq,
                          r->sc,  r->sq,  r->snu, r->spi, r->snu, r->spi,
                          r->snu, r->snu, r->snu, r->st,  r->st,  r->st};
    memcpy(s, v, sizeof v);
  }
}

/* Equilibrium moments, printed closed forms.
 * Q14: Eq. meq.  Q18: App. B equilibria. */
static void feq_cell(const model *m, double p, const double u[3], double *feq);

static void moment_equilibrium(const model *m, double p, const double u[3],
                               double *meq) {
  if (m->Q == 26) {
    /* no printed equilibria: m_eq = T f_eq, the definition (Eq. mrteqvT) */
    double feq[26];
    feq_cell(m, p, u, feq);
    for (int k = 0; k < 26; ++k) {
      double acc = 0.0;
      for (int a = 0; a < 26; ++a) acc += m->T[k * 26 + a] * feq[a];
      meq[k] = acc;
    }
    return;
  }
  const double ux = u[0], uy = u[1], uz = u[2];
  const double u2 = ux * ux + uy * uy + uz * uz;
  if (m->Q == 14) {
    meq[0] = 7.0 * p / 3.0 + u2 / 3.0;  /* P    */
    meq[1] = -7.0 * p + u2;             /* e    */
    meq[2] = ux;                        /* jx   */
    meq[3] = -7.0 * ux / 3.0;           /* qx   */
    meq[4] = uy;                        /* jy   */
    meq[5] = -7.0 * uy / 3.0;           /* qy   */
    meq[6] = uz;                        /* jz   */
    meq[7] = -7.0 * uz / 3.0;           /* qz   */
    meq[8] = 3.0 * ux * ux - u2;        /* 3pxx */
    meq[9] = uy * uy - uz * uz;         /* pww  */
    meq[10] = ux * uy;                  /* pxy  */
    meq[11] = uy * uz;                  /* pyz  */
    meq[12] = ux * uz;                  /* pxz  */
    meq[13] = 0.0;                      /* txyz */
  } else {
    meq[0] = 2.0 * p + 0.5 * u2;                    /* P     */
    meq[1] = -p + 0.5 * u2;                         /* e     */
    meq[2] = ux;                                    /* jx    */
    meq[3] = -2.0 * ux / 3.0;                       /* qx    */
    meq[4] = uy;                                    /* jy    */
    meq[5] = -2.0 * uy / 3.0;                       /* qy    */
    meq[6] = uz;                                    /* jz    */
    meq[7] = -2.0 * uz / 3.0;                       /* qz    */
    meq[8] = 3.0 * ux * ux - u2;                    /* 3pxx  */
    meq[9] = -0.5 * (3.0 * ux * ux - u2);           /* 3pixx */
    meq[10] = uy * uy - uz * uz;                    /* pww   */
    meq[11] = -0.5 * (uy * uy - uz * uz);           /* piww  */
    meq[12] = ux * uy;                              /* pxy   */
    meq[13] = uy * uz;                              /* pyz   */
    meq[14] = ux * uz;                              /* pxz   */
    meq[15] = 0.0;                                  /* tx    */
    meq[16] = 0.0;                                  /* ty    */
    meq[17] = 0.0;                                  /* tz    */
  }
}

/* Pressure from P and u, Eq. hgl with c_s^2 = 1/3:
 * p = c_s^2/(1-w0) [P - w0 |u|^2/(2 c_s^2)]. */
static double pressure(const model *m, double P, const double u[3]) {
  const double cs2 = 1.0 / 3.0;
  const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return cs2 / (1.0 - m->w0) * (P - m->w0 * u2 / (2.0 * cs2));
}

/* ---- one-cell collision ------------------------------------------------ */

static void collide_cell(const model *m, const double *s, const double *f,
                         const double F[3], double *fpost, double *u_out,
                         double *p_out) {
  const int Q = m->Q;
  double P = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < Q; ++a) {
    P += f[a];
    for (int d = 0; d < 3; ++d) j[d] += (double)m->c[a][d] * f[a];
  }
  double u[3];
  for (int d = 0; d < 3; ++d) u[d] = j[d] + 0.5 * F[d];
  const double p = pressure(m, P, u);

  /* m = T f */
  double mom[26];
  for (int k = 0; k < Q; ++k) {
    double acc = 0.0;
    for (int a = 0; a < Q; ++a) acc += (double)m->T[k * Q + a] * f[a];
    mom[k] = acc;
  }
  double meq[26];
  moment_equilibrium(m, p, u, meq);

  /* Guo source in velocity space, Fbar_a = w_a [3 c.F + 9 (c.u)(c.F) - 3 u.F],
   * projected with T; the P row is dropped. */
  double Fbar[26];
  const double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  for (int a = 0; a < Q; ++a) {
    const double cF = m->c[a][0] * F[0] + m->c[a][1] * F[1] + m->c[a][2] * F[2];
    const double cu = m->c[a][0] * u[0] + m->c[a][1] * u[1] + m->c[a][2] * u[2];
    Fbar[a] = m->w[a] * (3.0 * cF + 9.0 * cu * cF - 3.0 * uF);
  }
  double SF[26];
  for (int k = 0; k < Q; ++k) {
    double acc = 0.0;
    for (int a = 0; a < Q; ++a) acc += (double)m->T[k * Q + a] * Fbar[a];
    SF[k] = acc;
  }
  SF[0] = 0.0;

  double mpost[26];
  for (int k = 0; k < Q; ++k)
    mpost[k] = mom[k] - s[k] * (mom[k] - meq[k]) + (1.0 - 0.5 * s[k]) * SF[k];

  /* f* = T' D^-1 m* */
  for (int a = 0; a < Q; ++a) {
    double acc = 0.0;
    for (int k = 0; k < Q; ++k)
      acc += (double)m->T[k * Q + a] * (mpost[k] / m->D[k]);
    fpost[a] = acc;
  }
  if (u_out) memcpy(u_out, u, sizeof u);
  if (p_out) *p_out = p;
}

/* ---- geometry ------------------------------------------------------------ */

/* Face order: 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+. */
static int n_axis(const oracle_grid *g, int d) {
  return d == 0 ? g->nx : (d == 1 ? g->ny : g->nz);
}

/* Where does the pull source x - c_a of node (x,y,z) lie?  Returns 1 and the
 * source node if it is a fluid node (after periodic wraps and symmetry-plane
 * mirrors); returns 0 if it is a ghost node beyond a wall, and sets uw to
 * that ghost node's wall velocity: the velocity of the first moving face
 * (x-, x+, y-, y+, z-, z+ order) the ghost lies beyond, else zero (so
 * edge and corner ghosts of a lid layer count as lid).
 *
 * A symmetry face is a free-slip plane halfway between the last node and its
 * ghost layer: the ghost mirrors the node across the plane, so a source
 * beyond it is replaced by the mirrored node (the same coordinate as x along
 * that axis) and *mirror gets the axis bit (the population arriving at x
 * left that node with the normal component of its velocity reversed).  A
 * source beyond a wall on any axis is a wall link even if it also lies
 * beyond a symmetry face (the wall extends across the mirror plane). */
static int pull_source(const oracle_grid *g, const int xyz[3], const int c[3],
                       int src[3], double uw[3], int *mirror) {
  int beyond[6] = {0, 0, 0, 0, 0, 0};
  int solid = 0;
  *mirror = 0;
  for (int d = 0; d < 3; ++d) {
    const int n = n_axis(g, d);
    int v = xyz[d] - c[d];
    if (v < 0 || v >= n) {
      const int face = v < 0 ? 2 * d : 2 * d + 1;
      if (g->face[face] == ORACLE_PERIODIC) {
        v += v < 0 ? n : -n;
      } else if (g->face[face] == ORACLE_SYMMETRY) {
        v = xyz[d];
        *mirror |= 1 << d;
      } else {
        beyond[face] = 1;
        solid = 1;
      }
    }
    src[d] = v;
  }
  uw[0] = uw[1] = uw[2] = 0.0;
  if (!solid) {
    if (g->solid && g->solid[((int64_t)src[2] * g->ny + src[1]) * g->nx + src[0]])
      return 0; /* a solid node: bounce-back off a wall at rest */
    return 1;
  }
  for (int face = 0; face < 6; ++face) {
    if (beyond[face] && g->face[face] == ORACLE_MOVING_WALL) {
      double scale = 1.0;
      const int k = g->edge_axis[face] - 1;
      if (k >= 0 && k < 3) {
        if (xyz[k] == 0) scale = g->edge_scale[face][0];
        else if (xyz[k] == n_axis(g, k) - 1) scale = g->edge_scale[face][1];
      }
      uw[0] = g->u_wall[face][0] * scale;
      uw[1] = g->u_wall[face][1] * scale;
      uw[2] = g->u_wall[face][2] * scale;
      break;
    }
  }
  return 0;
}

/* The population whose velocity is c_a with the components of the axes in
 * `mask` reversed. */
static int mirrored(const model *m, int a, int mask) {
  if (!mask) return a;
  int c[3];
  for (int d = 0; d < 3; ++d) c[d] = (mask >> d) & 1 ? -m->c[a][d] : m->c[a][d];
  for (int b = 0; b < m->Q; ++b)
    if (m->c[b][0] == c[0] && m->c[b][1] == c[1] && m->c[b][2] == c[2]) return b;
  return a;  /* unreachable: both lattices are closed under axis reflections */
}

static double force_at(const oracle_params *prm, int64_t n, int d) {
  if (prm->period > 0.0)
    return prm->force[d] * cos(2.0 * M_PI * (double)n / prm->period);
  return prm->force[d];
}

static int is_neq(int kind) {
  return kind == ORACLE_NEQ_VELOCITY || kind == ORACLE_NEQ_PRESSURE;
}

static double face_pressure(const oracle_params *prm, int face, int64_t n) {
  if (prm->p_period > 0.0)
    return prm->p_face[face] + prm->p_amp[face] * cos(2.0 * M_PI * (double)n / prm->p_period);
  return prm->p_face[face];
}

/* Equilibrium populations, Eq. edf with lambda_a = w_a p / c_s^2 (c_s^2 = 1/3) */
static void feq_cell(const model *m, double p, const double u[3], double *feq) {
  const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int a = 0; a < m->Q; ++a) {
    const double cu = m->c[a][0] * u[0] + m->c[a][1] * u[1] + m->c[a][2] * u[2];
    feq[a] = m->w[a] * 3.0 * p + m->w[a] * (3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
  }
}

/* Non-equilibrium extrapolation of every node on an ORACLE_NEQ_* face, on
 * the pre-collision populations f of step n (in place).  The inward
 * neighbour x_f of a node is one node inward along the normal of every such
 * face the node lies on (diagonally inward on edges and corners); it is
 * never itself on such a face when those axes have at least 3 nodes, so the
 * order of the nodes does not matter.  A node on a velocity face takes the
 * velocity of the first such face in x-, x+, y-, y+, z-, z+ order and the
 * pressure of x_f; a node only on pressure faces takes the pressure of the
 * first one and the velocity of x_f. */
static void neq_extrapolate(const model *m, const oracle_grid *g, const oracle_params *prm,
                            int64_t n, double *f) {
  const int Q = m->Q, nx = g->nx, ny = g->ny, nz = g->nz;
  const int64_t N = (int64_t)nx * ny * nz;
  const double F[3] = {force_at(prm, n, 0), force_at(prm, n, 1), force_at(prm, n, 2)};
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int xyz[3] = {x, y, z};
        int xf[3] = {x, y, z};
        int vel_face = -1, pre_face = -1;
        for (int d = 0; d < 3; ++d) {
          const int nd = n_axis(g, d);
          for (int side = 0; side < 2; ++side) {
            const int face = 2 * d + side;
            const int on = side == 0 ? xyz[d] == 0 : xyz[d] == nd - 1;
            if (!on || !is_neq(g->face[face])) continue;
            xf[d] = side == 0 ? 1 : nd - 2;
            if (g->face[face] == ORACLE_NEQ_VELOCITY && vel_face < 0) vel_face = face;
            if (g->face[face] == ORACLE_NEQ_PRESSURE && pre_face < 0) pre_face = face;
          }
        }
        if (vel_face < 0 && pre_face < 0) continue;
        const int64_t ib = ((int64_t)z * ny + y) * nx + x;
        const int64_t jf = ((int64_t)xf[2] * ny + xf[1]) * nx + xf[0];
        double P = 0.0, uf[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < Q; ++a) {
          P += f[a * N + jf];
          for (int d = 0; d < 3; ++d) uf[d] += (double)m->c[a][d] * f[a * N + jf];
        }
        for (int d = 0; d < 3; ++d) uf[d] += 0.5 * F[d];
        const double pf = pressure(m, P, uf);
        double ub[3], pb;
        for (int d = 0; d < 3; ++d) ub[d] = vel_face >= 0 ? g->u_wall[vel_face][d] : uf[d];
        pb = pre_face >= 0 ? face_pressure(prm, pre_face, n) : pf;
        double eb[26], ef[26];
        feq_cell(m, pb, ub, eb);
        feq_cell(m, pf, uf, ef);
        for (int a = 0; a < Q; ++a) f[a * N + ib] = eb[a] + (f[a * N + jf] - ef[a]);
      }
}

/* ---- public entry points --------------------------------------------------- */

int oracle_velocities(int Q, int *c_out) {
  model m;
  if (model_init(Q, &m)) return -1;
  for (int a = 0; a < Q; ++a)
    for (int d = 0; d < 3; ++d) c_out[3 * a + d] = m.c[a][d];
  return 0;
}

int oracle_weights(int Q, double *w_out, double *w0_out) {
  model m;
  if (model_init(Q, &m)) return -1;
  for (int a = 0; a < Q; ++a) w_out[a] = m.w[a];
  *w0_out = m.w0;
  return 0;
}

int oracle_transform(int Q, double *T_out) {
  model m;
  if (model_init(Q, &m)) return -1;
  memcpy(T_out, m.T, sizeof(double) * Q * Q);
  return 0;
}

int oracle_moment_equilibrium(int Q, double p, const double *u, double *meq) {
  model m;
  if (model_init(Q, &m)) return -1;
  moment_equilibrium(&m, p, u, meq);
  return 0;
}

int oracle_pressure(int Q, double P, const double *u, double *p) {
  model m;
  if (model_init(Q, &m)) return -1;
  *p = pressure(&m, P, u);
  return 0;
}

int oracle_feq(int Q, double p, const double *u, double *feq) {
  model m;
  if (model_init(Q, &m)) return -1;
  /* Eq. edf with lambda_a = w_a p / c_s^2 for a >= 1 (Eq. lamda_alpha) */
  const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int a = 0; a < Q; ++a) {
    const double cu = m.c[a][0] * u[0] + m.c[a][1] * u[1] + m.c[a][2] * u[2];
    feq[a] = m.w[a] * 3.0 * p +
             m.w[a] * (3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
  }
  return 0;
}

int oracle_collide(int Q, const oracle_rates *r, const double *f,
                   const double *F, double *fpost) {
  model m;
  if (model_init(Q, &m)) return -1;
  double s[26];
  relaxation_diag(&m, r, s);
  collide_cell(&m, s, f, F, fpost, NULL, NULL);
  return 0;
}

int oracle_init_equilibrium(const oracle_grid *g, const double *u,
                            const double *p, double *f) {
  model m;
  if (model_init(g->Q, &m)) return -1;
  const int64_t N = (int64_t)g->nx * g->ny * g->nz;
  for (int64_t i = 0; i < N; ++i) {
    double ui[3] = {0.0, 0.0, 0.0};
    if (u)
      for (int d = 0; d < 3; ++d) ui[d] = u[d * N + i];
    const double pi = p ? p[i] : 0.0;
    double feq[26];
    oracle_feq(g->Q, pi, ui, feq);
    const int solid = g->solid && g->solid[i];
    for (int a = 0; a < g->Q; ++a) f[a * N + i] = solid ? 0.0 : feq[a];
  }
  return 0;
}

int oracle_step(const oracle_grid *g, const oracle_params *prm, int64_t n,
                const double *f_in, double *f_out, int nthreads) {
  model m;
  if (model_init(g->Q, &m)) return -1;
  const int Q = m.Q;
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const int64_t N = (int64_t)nx * ny * nz;
  for (int d = 0; d < 3; ++d)
    if ((is_neq(g->face[2 * d]) || is_neq(g->face[2 * d + 1])) && n_axis(g, d) < 3)
      return -3; /* an extrapolation boundary needs an inward neighbour */
  for (int face = 0; face < 6; ++face)
    if (g->solid && is_neq(g->face[face])) return -4; /* not combined */
  double s[26];
  relaxation_diag(&m, &prm->rates, s);
  int opp[26];
  for (int a = 0; a < Q; ++a) opp[a] = opposite(&m, a);
  const double F[3] = {force_at(prm, n, 0), force_at(prm, n, 1),
                       force_at(prm, n, 2)};

  /* post-collision populations of every node, then pull streaming */
  double *fpost = (double *)malloc(sizeof(double) * Q * N);
  if (!fpost) return -2;

#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
  for (int z = 0; z < nz; ++z) {
    double fc[26], fp[26];
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t i = ((int64_t)z * ny + y) * nx + x;
        if (g->solid && g->solid[i]) {
          for (int a = 0; a < Q; ++a) fpost[a * N + i] = 0.0;
          continue;
        }
        for (int a = 0; a < Q; ++a) fc[a] = f_in[a * N + i];
        collide_cell(&m, s, fc, F, fp, NULL, NULL);
        for (int a = 0; a < Q; ++a) fpost[a * N + i] = fp[a];
      }
  }

#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
  for (int z = 0; z < nz; ++z) {
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int xyz[3] = {x, y, z};
        const int64_t i = ((int64_t)z * ny + y) * nx + x;
        if (g->solid && g->solid[i]) {
          for (int a = 0; a < Q; ++a) f_out[a * N + i] = 0.0;
          continue;
        }
        for (int a = 0; a < Q; ++a) {
          int src[3], mirror;
          double uw[3];
          if (pull_source(g, xyz, m.c[a], src, uw, &mirror)) {
            const int64_t j = ((int64_t)src[2] * ny + src[1]) * nx + src[0];
            f_out[a * N + i] = fpost[mirrored(&m, a, mirror) * N + j];
          } else {
            const double cu =
                m.c[a][0] * uw[0] + m.c[a][1] * uw[1] + m.c[a][2] * uw[2];
            f_out[a * N + i] = fpost[opp[a] * N + i] + 6.0 * m.w[a] * cu;
          }
        }
      }
  }
  free(fpost);
  int any_neq = 0;
  for (int face = 0; face < 6; ++face) any_neq |= is_neq(g->face[face]);
  if (any_neq) neq_extrapolate(&m, g, prm, n + 1, f_out);
  return 0;
}

int oracle_run(const oracle_grid *g, const oracle_params *prm, int64_t n0,
               int64_t nsteps, double *f, int nthreads) {
  const int64_t N = (int64_t)g->nx * g->ny * g->nz;
  double *tmp = (double *)malloc(sizeof(double) * g->Q * N);
  if (!tmp) return -2;
  for (int64_t k = 0; k < nsteps; ++k) {
    int rc = oracle_step(g, prm, n0 + k, f, tmp, nthreads);
    if (rc) {
      free(tmp);
      return rc;
    }
    memcpy(f, tmp, sizeof(double) * g->Q * N);
  }
  free(tmp);
  return 0;
}

int oracle_macroscopic(const oracle_grid *g, const oracle_params *prm,
                       int64_t n, const double *f, double *u, double *p) {
  model m;
  if (model_init(g->Q, &m)) return -1;
  const int64_t N = (int64_t)g->nx * g->ny * g->nz;
  const double F[3] = {force_at(prm, n, 0), force_at(prm, n, 1),
                       force_at(prm, n, 2)};
  for (int64_t i = 0; i < N; ++i) {
    if (g->solid && g->solid[i]) {
      if (u)
        for (int d = 0; d < 3; ++d) u[d * N + i] = 0.0;
      if (p) p[i] = 0.0;
      continue;
    }
    double P = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < m.Q; ++a) {
      P += f[a * N + i];
      for (int d = 0; d < 3; ++d) j[d] += (double)m.c[a][d] * f[a * N + i];
    }
    double ui[3];
    for (int d = 0; d < 3; ++d) ui[d] = j[d] + 0.5 * F[d];
    if (u)
      for (int d = 0; d < 3; ++d) u[d * N + i] = ui[d];
    if (p) p[i] = pressure(&m, P, ui);
  }
  return 0;
}
