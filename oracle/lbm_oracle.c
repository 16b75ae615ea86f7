/*
 * lbm_oracle.c -- plain FP64 CPU oracle for the D3Q19 BGK lattice Boltzmann method
 * with the on-site velocity boundary condition of Hecht & Harting, "Implementation
 * of on-site velocity boundary conditions for D3Q19 lattice Boltzmann"
 * (arXiv:0811.4593).
 *
 * TEST INFRASTRUCTURE. This is the slow, obviously-correct statement of what the
 * CUDA library computes. It shares no code, header or table with that library and
 * the library never calls it; only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.
 *
 * Conventions
 *   - population f_i (i = 1..19, the paper's numbering) lives at array index i-1;
 *     the F(i) macro below reads and writes it by the paper's index;
 *   - lattice arrays are [19][nz][ny][nx] with x fastest;
 *   - faces: 0: x=0, 1: x=nx-1, 2: y=0, 3: y=ny-1, 4: z=0, 5: z=nz-1; a face's
 *     inward normal is +e_a for the low face and -e_a for the high face of axis a;
 *   - a velocity face (kind 1) carries a table of prescribed velocities [n2][n1][3],
 *     where (t1, t2) are the two tangential axes in increasing axis order; v = 0 is
 *     no-slip. A pressure face (kind 2) carries a density table [n2][n1] and a velocity
 *     table whose tangential part is prescribed (its normal part is ignored);
 *   - an axis is periodic when both of its faces are periodic (kind 0); otherwise each
 *     of its faces is a velocity or a pressure face. Pressure faces lie on one axis at
 *     most, so an edge or corner borders at most one pressure plane;
 *   - every sum over populations runs in index order i = 1..19.
 *
 * Readings of the paper where it is ambiguous or garbled (all other steps follow the
 * equations cited at each function):
 *   R1 Sec. "General on-site velocity boundary condition", eq. bbshort: the compact
 *      rule prints the coefficient rho/6 for every population; the explicit
 *      per-plane formulas (eq. f5: rho v_z / 3 for the normal population) require
 *      6 w_i, i.e. rho/3 for axis and rho/6 for diagonal populations. Used here.
 *   R2 Sec. "On-site no-slip boundary condition", eq. edge: taken literally, adding
 *      N c_i.t_i doubles the slip along the edge. The sign that removes it is used:
 *      f_i = f_-i - (c_i.e) (f_{+e} - f_{-e}) / 4 for every unknown, non-buried i,
 *      where e is the edge direction.
 *   R3 eq. buried: the sum runs over the 16 moving populations that are not the two
 *      buried links (6 axis + 10 diagonal, total weight 22/36), after bounce-back.
 *   R4 eq. corner: the sum runs over the 12 moving populations with
 *      c_i.(n1+n2+n3) != 0 (6 axis + 6 diagonal, total weight 18/36).
 *   R5 edges and corners always take v = 0 (the no-slip rule "can be used on all
 *      edges" when the in/outflow profile decays to zero there).
 *   R6 a time step is: pull streaming, boundary closure on the unknown populations,
 *      then BGK collision; the initial state counts as post-collision.
 *   R7 appendix, back plane: the velocity form of the density relation is printed
 *      for v_x; the back plane's normal velocity is v_y.
 *   R8 pressure planes: edges and corners next to one take the buried-link values
 *      that make their density the prescribed one (eq. buried_rho, corner variant);
 *      the along-edge momentum correction is the same as for velocity planes.
 *   R9 convex edges (eq. edge2): after bounce-back of the population whose source is
 *      solid, N_i is subtracted from every population travelling into the bulk
 *      (c_i.d > 0, d the edge's bulk normal); the four of them with c_i.e != 0 carry
 *      the whole along-edge momentum away.
 *   R10 edge/plane junctions: the rest population is printed as 12/36 of the sum of
 *      the 18 moving populations, which at rest would remove a ninth of the node's
 *      density every step; it is read as 12/36 of the node density, i.e. one half of
 *      the sum of the moving populations. Only convex edges meet a plane this way: a
 *      concave edge ending on a perpendicular plane is a corner (eq. corner).
 *   R11 body force (eq. gravity): the equilibrium of the collision takes the velocity
 *      u + tau F / rho; the reported velocity is that of the stored post-collision
 *      state, u + F / rho.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* Lattice vectors: c_i is the i-th column of the matrix M (eq. deffs). */
static const int CV[Q][3] = {
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1}, /* c1..c6 */
    {1, 1, 0},  {1, -1, 0}, {1, 0, 1},  {1, 0, -1},                         /* c7..c10 */
    {-1, 1, 0}, {-1, -1, 0}, {-1, 0, 1}, {-1, 0, -1},                       /* c11..c14 */
    {0, 1, 1},  {0, 1, -1}, {0, -1, 1}, {0, -1, -1},                        /* c15..c18 */
    {0, 0, 0}};                                                             /* c19 */

/* Lattice weights (eq. weights). */
static const double WT[Q] = {2.0 / 36, 2.0 / 36, 2.0 / 36, 2.0 / 36, 2.0 / 36, 2.0 / 36,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                             12.0 / 36};

#define F(i) f[(i)-1]

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_UNFILLED = 2 };

static int dot_ci(int k, const int n[3]) { return CV[k][0] * n[0] + CV[k][1] * n[1] + CV[k][2] * n[2]; }
static double dot_cv(int k, const double v[3]) { return CV[k][0] * v[0] + CV[k][1] * v[1] + CV[k][2] * v[2]; }

/* Index of the population with c = -c_k, found by search. */
static int opposite(int k) {
  for (int m = 0; m < Q; ++m)
    if (CV[m][0] == -CV[k][0] && CV[m][1] == -CV[k][1] && CV[m][2] == -CV[k][2]) return m;
  return -1;
}

/* Inward normal of face 0..5. */
static void face_normal(int face, int n[3]) {
  n[0] = n[1] = n[2] = 0;
  n[face / 2] = (face % 2 == 0) ? 1 : -1;
}

/* ----------------------------------------------------------------------------------
 * Equilibrium and moments.
 * -------------------------------------------------------------------------------- */

/* Second-order equilibrium (eq. feq) with c_s^2 = 1/3. */
void orc_feq(double rho, const double* v, double* feq) {
  const double cs2 = 1.0 / 3.0;
  double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  for (int k = 0; k < Q; ++k) {
    double cv = dot_cv(k, v);
    feq[k] = WT[k] * rho * (1.0 + cv / cs2 + cv * cv / (2.0 * cs2 * cs2) - vv / (2.0 * cs2));
  }
}

/* Density (eq. rho) and velocity (eq. vel); out = {rho, v_x, v_y, v_z}. */
void orc_moments(const double* f, double* out) {
  double rho = 0, j[3] = {0, 0, 0};
  for (int k = 0; k < Q; ++k) {
    rho += f[k];
    for (int a = 0; a < 3; ++a) j[a] += f[k] * CV[k][a];
  }
  out[0] = rho;
  for (int a = 0; a < 3; ++a) out[a + 1] = j[a] / rho;
}

/* BGK collision (eq. bgk): f <- f - (f - f_eq(rho, v)) / tau. */
void orc_collide(double* f, double tau) {
  double m[4], feq[Q];
  orc_moments(f, m);
  orc_feq(m[0], m + 1, feq);
  for (int k = 0; k < Q; ++k) f[k] = f[k] - (f[k] - feq[k]) / tau;
}

/* BGK collision under a body force F (eq. gravity, reading R11): the equilibrium
 * takes the velocity v + tau F / rho. */
void orc_collide_force(double* f, double tau, const double* force) {
  double m[4], feq[Q], v[3];
  orc_moments(f, m);
  for (int a = 0; a < 3; ++a) v[a] = m[a + 1] + tau * force[a] / m[0];
  orc_feq(m[0], v, feq);
  for (int k = 0; k < Q; ++k) f[k] = f[k] - (f[k] - feq[k]) / tau;
}

/* ----------------------------------------------------------------------------------
 * Face closure, form (i): the explicit per-plane formulas. Each returns rho and
 * overwrites the five unknown populations; v is the velocity of the node in lattice
 * axes. rho_fixed > 0 is a density given in advance (the pressure variant); otherwise
 * rho comes from the plane's density relation.
 * -------------------------------------------------------------------------------- */

/* Bottom plane z = 0: eq. uin, eq. f5, eq. f9-f17, eq. Nx, eq. Ny. */
static double close_bottom(double* f, const double* v, double rho_fixed) {
  double rho = rho_fixed > 0.0 ? rho_fixed : (F(1) + F(2) + F(3) + F(4) + F(7) + F(8) + F(11) + F(12) + F(19) +
                2.0 * (F(6) + F(10) + F(14) + F(16) + F(18))) / (1.0 - v[2]);
  double Nx = 0.5 * (F(1) + F(7) + F(8) - (F(2) + F(11) + F(12))) - rho * v[0] / 3.0;
  double Ny = 0.5 * (F(3) + F(7) + F(11) - (F(4) + F(8) + F(12))) - rho * v[1] / 3.0;
  F(5) = F(6) + rho * v[2] / 3.0;
  F(9) = F(14) + rho / 6.0 * (v[2] + v[0]) - Nx;
  F(13) = F(10) + rho / 6.0 * (v[2] - v[0]) + Nx;
  F(15) = F(18) + rho / 6.0 * (v[2] + v[1]) - Ny;
  F(17) = F(16) + rho / 6.0 * (v[2] - v[1]) + Ny;
  return rho;
}

/* Top plane z = nz-1: appendix, top plane. */
static double close_top(double* f, const double* v, double rho_fixed) {
  double rho = rho_fixed > 0.0 ? rho_fixed : (F(1) + F(2) + F(3) + F(4) + F(7) + F(11) + F(12) + F(8) + F(19) +
                2.0 * (F(5) + F(9) + F(13) + F(15) + F(17))) / (v[2] + 1.0);
  double Nx = 0.5 * (F(1) + F(7) + F(8) - (F(2) + F(11) + F(12))) - rho * v[0] / 3.0;
  double Ny = 0.5 * (F(3) + F(7) + F(11) - (F(4) + F(8) + F(12))) - rho * v[1] / 3.0;
  F(6) = F(5) - rho * v[2] / 3.0;
  F(10) = F(13) + rho / 6.0 * (-v[2] + v[0]) - Nx;
  F(14) = F(9) + rho / 6.0 * (-v[2] - v[0]) + Nx;
  F(16) = F(17) + rho / 6.0 * (-v[2] + v[1]) - Ny;
  F(18) = F(15) + rho / 6.0 * (-v[2] - v[1]) + Ny;
  return rho;
}

/* Left plane x = 0: appendix, eq. rhooutx, eq. Nxy, eq. Nxz. */
static double close_left(double* f, const double* v, double rho_fixed) {
  double rho = rho_fixed > 0.0 ? rho_fixed : (F(3) + F(4) + F(5) + F(6) + F(15) + F(16) + F(17) + F(18) + F(19) +
                2.0 * (F(2) + F(11) + F(12) + F(13) + F(14))) / (1.0 - v[0]);
  double Ny = 0.5 * (F(3) + F(15) + F(16) - (F(4) + F(17) + F(18))) - rho * v[1] / 3.0;
  double Nz = 0.5 * (F(5) + F(17) + F(15) - (F(6) + F(16) + F(18))) - rho * v[2] / 3.0;
  F(1) = F(2) + rho * v[0] / 3.0;
  F(8) = F(11) + rho / 6.0 * (v[0] - v[1]) + Ny;
  F(7) = F(12) + rho / 6.0 * (v[0] + v[1]) - Ny;
  F(9) = F(14) + rho / 6.0 * (v[0] + v[2]) - Nz;
  F(10) = F(13) + rho / 6.0 * (v[0] - v[2]) + Nz;
  return rho;
}

/* Right plane x = nx-1: appendix, eq. rhoinx. */
static double close_right(double* f, const double* v, double rho_fixed) {
  double rho = rho_fixed > 0.0 ? rho_fixed : (F(3) + F(4) + F(5) + F(6) + F(15) + F(16) + F(17) + F(18) + F(19) +
                2.0 * (F(1) + F(7) + F(8) + F(9) + F(10))) / (v[0] + 1.0);
  double Ny = 0.5 * (F(3) + F(15) + F(16) - (F(4) + F(17) + F(18))) - rho * v[1] / 3.0;
  double Nz = 0.5 * (F(5) + F(17) + F(15) - (F(6) + F(16) + F(18))) - rho * v[2] / 3.0;
  F(2) = F(1) - rho * v[0] / 3.0;
  F(11) = F(8) + rho / 6.0 * (-v[0] + v[1]) - Ny;
  F(12) = F(7) + rho / 6.0 * (-v[0] - v[1]) + Ny;
  F(14) = F(9) + rho / 6.0 * (-v[0] - v[2]) + Nz;
  F(13) = F(10) + rho / 6.0 * (-v[0] + v[2]) - Nz;
  return rho;
}

/* Front plane y = 0: appendix, eq. rhoiny, eq. Nyx, eq. Nyz. */
static double close_front(double* f, const double* v, double rho_fixed) {
  double rho = rho_fixed > 0.0 ? rho_fixed : (F(1) + F(2) + F(5) + F(6) + F(9) + F(10) + F(13) + F(14) + F(19) +
                2.0 * (F(4) + F(8) + F(12) + F(17) + F(18))) / (1.0 - v[1]);
  double Nx = 0.5 * (F(1) + F(9) + F(10) - (F(2) + F(13) + F(14))) - rho * v[0] / 3.0;
  double Nz = 0.5 * (F(5) + F(9) + F(13) - (F(6) + F(10) + F(14))) - rho * v[2] / 3.0;
  F(3) = F(4) + rho * v[1] / 3.0;
  F(7) = F(12) + rho / 6.0 * (v[1] + v[0]) - Nx;
  F(11) = F(8) + rho / 6.0 * (v[1] - v[0]) + Nx;
  F(15) = F(18) + rho / 6.0 * (v[1] + v[2]) - Nz;
  F(16) = F(17) + rho / 6.0 * (v[1] - v[2]) + Nz;
  return rho;
}

/* Back plane y = ny-1: appendix, eq. rhoouty (velocity form; the printed v_x of the
 * density-given variant is read as v_y, which this velocity form does not use). */
static double close_back(double* f, const double* v, double rho_fixed) {
  double rho = rho_fixed > 0.0 ? rho_fixed : (F(1) + F(2) + F(5) + F(6) + F(9) + F(10) + F(13) + F(14) + F(19) +
                2.0 * (F(3) + F(7) + F(11) + F(15) + F(16))) / (v[1] + 1.0);
  double Nx = 0.5 * (F(1) + F(9) + F(10) - (F(2) + F(13) + F(14))) - rho * v[0] / 3.0;
  double Nz = 0.5 * (F(5) + F(9) + F(13) - (F(6) + F(10) + F(14))) - rho * v[2] / 3.0;
  F(4) = F(3) - rho * v[1] / 3.0;
  F(12) = F(7) + rho / 6.0 * (-v[1] - v[0]) + Nx;
  F(8) = F(11) + rho / 6.0 * (-v[1] + v[0]) - Nx;
  F(18) = F(15) + rho / 6.0 * (-v[1] - v[2]) + Nz;
  F(17) = F(16) + rho / 6.0 * (-v[1] + v[2]) - Nz;
  return rho;
}

/* ----------------------------------------------------------------------------------
 * Face closure, form (ii): the compact rule for any plane (eq. bbshort, reading R1).
 * For every population i pointing out of the domain (c_i.n < 0) the population -i
 * pointing in is
 *   f_-i = f_i - 6 w_i rho c_i.v - (rho/3) t_i.v + 1/2 sum_j f_j (t_i.c_j)(1 - |c_j.n|)
 * with t_i = c_i - (c_i.n) n and rho from the plane's density relation (eq. uin).
 * -------------------------------------------------------------------------------- */
/* zero_n != 0 is the comparison closure of the paper's Fig. (vdifffields) b: the same
 * non-equilibrium bounce-back with the transverse corrections N forced to zero
 * (eqs. f9NoNs-f17NoNs), used only to reproduce that comparison. */
static double close_face_compact(double* f, int face, const double* v, double rho_fixed, int zero_n) {
  int n[3];
  face_normal(face, n);
  /* density: in-plane populations once, outgoing ones twice, unknown ones not at all */
  double s = 0.0;
  for (int k = 0; k < Q; ++k) {
    int cn = dot_ci(k, n);
    if (cn == 0) s += f[k];
    else if (cn < 0) s += 2.0 * f[k];
  }
  double vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
  double rho = rho_fixed > 0.0 ? rho_fixed : s / (1.0 - vn);
  for (int k = 0; k < Q; ++k) {
    int cn = dot_ci(k, n);
    if (cn >= 0) continue; /* only outgoing i */
    double t[3];
    for (int a = 0; a < 3; ++a) t[a] = CV[k][a] - cn * n[a];
    double tv = t[0] * v[0] + t[1] * v[1] + t[2] * v[2];
    double corr = 0.0; /* sum over in-plane j; the factor (1-|c_j.n|) drops the rest */
    for (int j = 0; j < Q; ++j) {
      if (dot_ci(j, n) != 0) continue;
      double tc = t[0] * CV[j][0] + t[1] * CV[j][1] + t[2] * CV[j][2];
      corr += f[j] * tc;
    }
    if (zero_n) f[opposite(k)] = f[k] - 6.0 * WT[k] * rho * dot_cv(k, v);
    else f[opposite(k)] = f[k] - 6.0 * WT[k] * rho * dot_cv(k, v) - rho / 3.0 * tv + 0.5 * corr;
  }
  return rho;
}

/* form: bit 0 set = compact rule, else the explicit per-plane formulas; bit 1 set = the
 * N = 0 comparison closure (compact rule only). */
static double close_face_form(int face, int form, double* f, const double* v, double rho_fixed) {
  if (form & 1) return close_face_compact(f, face, v, rho_fixed, form & 2);
  switch (face) {
    case 0: return close_left(f, v, rho_fixed);
    case 1: return close_right(f, v, rho_fixed);
    case 2: return close_front(f, v, rho_fixed);
    case 3: return close_back(f, v, rho_fixed);
    case 4: return close_bottom(f, v, rho_fixed);
    default: return close_top(f, v, rho_fixed);
  }
}

/* Entry for both forms: form 0 = explicit per-plane formulas, form 1 = compact rule. */
int orc_close_face(int face, int form, double* f, const double* v, double* rho_out) {
  if (face < 0 || face > 5) return ORC_ERR_ARG;
  double rho = close_face_form(face, form, f, v, -1.0);
  if (rho_out) *rho_out = rho;
  return ORC_OK;
}

/* ----------------------------------------------------------------------------------
 * Pressure (density) variant of the face closure (Sec. "General on-site velocity
 * boundary condition", eq. rhoin; appendix: top plane, eq. voutx, eq. uinx, eq. uiny,
 * eq. uouty). The density rho0 and the tangential velocity are prescribed; the normal
 * velocity follows from the plane's density relation; the unknown populations then
 * follow the same rules as for the velocity closure with rho = rho0.
 * -------------------------------------------------------------------------------- */

/* Velocity component along the plane's axis, explicit per-plane relations (form 0). */
static double pressure_velocity_explicit(int face, const double* f, double rho0) {
  switch (face) {
    case 4: /* bottom, eq. rhoin */
      return 1.0 - (F(1) + F(2) + F(3) + F(4) + F(7) + F(8) + F(11) + F(12) + F(19) +
                    2.0 * (F(6) + F(10) + F(14) + F(16) + F(18))) / rho0;
    case 5: /* top */
      return -1.0 + (F(1) + F(2) + F(3) + F(4) + F(7) + F(11) + F(12) + F(8) + F(19) +
                     2.0 * (F(5) + F(9) + F(13) + F(15) + F(17))) / rho0;
    case 0: /* left, eq. voutx */
      return 1.0 - (F(3) + F(4) + F(5) + F(6) + F(15) + F(16) + F(17) + F(18) + F(19) +
                    2.0 * (F(2) + F(11) + F(12) + F(13) + F(14))) / rho0;
    case 1: /* right, eq. uinx */
      return -1.0 + (F(3) + F(4) + F(5) + F(6) + F(15) + F(16) + F(17) + F(18) + F(19) +
                     2.0 * (F(1) + F(7) + F(8) + F(9) + F(10))) / rho0;
    case 2: /* front, eq. uiny */
      return 1.0 - (F(1) + F(2) + F(5) + F(6) + F(9) + F(10) + F(13) + F(14) + F(19) +
                    2.0 * (F(4) + F(8) + F(12) + F(17) + F(18))) / rho0;
    default: /* back, eq. uouty (its printed v_x read as v_y) */
      return -1.0 + (F(1) + F(2) + F(5) + F(6) + F(9) + F(10) + F(13) + F(14) + F(19) +
                     2.0 * (F(3) + F(7) + F(11) + F(15) + F(16))) / rho0;
  }
}

/* Same from the general relation u.n = 1 - (sum in-plane + 2 sum outgoing) / rho0 (form 1). */
static double pressure_velocity_compact(int face, const double* f, double rho0) {
  int n[3];
  face_normal(face, n);
  double s = 0.0;
  for (int k = 0; k < Q; ++k) {
    int cn = dot_ci(k, n);
    if (cn == 0) s += f[k];
    else if (cn < 0) s += 2.0 * f[k];
  }
  return (double)n[face / 2] * (1.0 - s / rho0);
}

/* Pressure closure: v holds the tangential velocity (its normal component is ignored);
 * the normal component found is returned in *vn_out (along the plane's axis). */
int orc_close_face_pressure(int face, int form, double* f, double rho0, const double* v, double* vn_out) {
  if (face < 0 || face > 5 || !(rho0 > 0.0)) return ORC_ERR_ARG;
  double u[3] = {v[0], v[1], v[2]};
  double vn = (form & 1) ? pressure_velocity_compact(face, f, rho0) : pressure_velocity_explicit(face, f, rho0);
  u[face / 2] = vn;
  close_face_form(face, form, f, u, rho0);
  if (vn_out) *vn_out = vn;
  return ORC_OK;
}

/* ----------------------------------------------------------------------------------
 * Concave edge, no-slip (Sec. "On-site no-slip boundary condition", eq. Nxzy,
 * eq. edge, eq. buried; readings R2, R3). n1, n2 are the inward normals of the
 * two planes meeting at the edge.
 * -------------------------------------------------------------------------------- */
static void close_edge_normals(double* f, const int n1[3], const int n2[3], double rho_p) {
  int e[3] = {n1[1] * n2[2] - n1[2] * n2[1], n1[2] * n2[0] - n1[0] * n2[2],
              n1[0] * n2[1] - n1[1] * n2[0]};
  int buried[Q], unknown[Q];
  for (int k = 0; k < Q; ++k) {
    int d = 1, m = 1;
    for (int a = 0; a < 3; ++a) {
      if (CV[k][a] != n1[a] - n2[a]) d = 0;
      if (CV[k][a] != n2[a] - n1[a]) m = 0;
    }
    buried[k] = d || m;
    unknown[k] = dot_ci(k, n1) > 0 || dot_ci(k, n2) > 0;
  }
  /* 1. bounce back every unknown population that is not a buried link */
  for (int k = 0; k < Q; ++k)
    if (unknown[k] && !buried[k]) f[k] = f[opposite(k)];
  /* 2. remove the momentum left along the edge: N = 1/4 sum_j f_j (c_j.e) over the
   *    populations lying in both planes (eq. Nxzy, eq. edge) */
  double Ne = 0.0;
  for (int j = 0; j < Q; ++j) {
    if (dot_ci(j, n1) != 0 || dot_ci(j, n2) != 0) continue;
    Ne += f[j] * dot_ci(j, e);
  }
  Ne *= 0.25;
  for (int k = 0; k < Q; ++k)
    if (unknown[k] && !buried[k]) f[k] -= dot_ci(k, e) * Ne;
  /* 3. buried links and rest population (eq. buried); next to a pressure plane the
   *    node density is the prescribed rho_p (eq. buried_rho) */
  double s = 0.0;
  for (int k = 0; k < Q - 1; ++k)
    if (!buried[k]) s += f[k];
  double fb = s / 22.0;
  if (rho_p > 0.0) fb = (rho_p - 22.0 * fb) / 14.0;
  for (int k = 0; k < Q - 1; ++k)
    if (buried[k]) f[k] = fb;
  F(19) = 12.0 * fb;
}

/* rho_p > 0: the edge borders a pressure plane of density rho_p. */
int orc_close_edge(int face_a, int face_b, double* f, double rho_p) {
  if (face_a < 0 || face_a > 5 || face_b < 0 || face_b > 5 || face_a / 2 == face_b / 2) return ORC_ERR_ARG;
  int n1[3], n2[3];
  face_normal(face_a, n1);
  face_normal(face_b, n2);
  close_edge_normals(f, n1, n2, rho_p);
  return ORC_OK;
}

/* ----------------------------------------------------------------------------------
 * Corner, no-slip (eq. corner, reading R4).
 * -------------------------------------------------------------------------------- */
static void close_corner_normals(double* f, const int n1[3], const int n2[3], const int n3[3], double rho_p) {
  int s3[3] = {n1[0] + n2[0] + n3[0], n1[1] + n2[1] + n3[1], n1[2] + n2[2] + n3[2]};
  int buried[Q], unknown[Q];
  for (int k = 0; k < Q; ++k) {
    buried[k] = (k < Q - 1) && dot_ci(k, s3) == 0;
    unknown[k] = dot_ci(k, n1) > 0 || dot_ci(k, n2) > 0 || dot_ci(k, n3) > 0;
  }
  for (int k = 0; k < Q; ++k)
    if (unknown[k] && !buried[k]) f[k] = f[opposite(k)];
  double s = 0.0;
  for (int k = 0; k < Q - 1; ++k)
    if (!buried[k]) s += f[k];
  double fb = s / 18.0;
  if (rho_p > 0.0) fb = rho_p / 18.0 - fb; /* next to a pressure plane */
  for (int k = 0; k < Q - 1; ++k)
    if (buried[k]) f[k] = fb;
  F(19) = 12.0 * fb;
}

/* rho_p > 0: the corner borders a pressure plane of density rho_p. */
int orc_close_corner(int face_x, int face_y, int face_z, double* f, double rho_p) {
  if (face_x < 0 || face_x > 1 || face_y < 2 || face_y > 3 || face_z < 4 || face_z > 5) return ORC_ERR_ARG;
  int n1[3], n2[3], n3[3];
  face_normal(face_x, n1);
  face_normal(face_y, n2);
  face_normal(face_z, n3);
  close_corner_normals(f, n1, n2, n3, rho_p);
  return ORC_OK;
}

/* ----------------------------------------------------------------------------------
 * Boundary nodes of a general geometry (Sec. "On-site no-slip boundary condition",
 * complex geometries): the normal is stored on the node as an integer code.
 *   1..6      plane, inward normal c_code (eq. bbshort with v = 0)
 *   7..18     concave edge whose bulk normal is the diagonal c_code (eq. edge)
 *   -18..-7   convex edge whose bulk normal is the diagonal c_-code (eq. edge2)
 *   19..26    corner with bulk normal (sx, sy, sz), code = 19 + [sx<0] + 2[sy<0] + 4[sz<0]
 *             (eq. corner)
 *   27..50    junction of a convex edge with the plane perpendicular to it:
 *             code = 27 + 4 (p - 1) + j, plane normal c_p (p = 1..6), edge bulk normal
 *             the j-th (j = 0..3, increasing index) diagonal c_i with c_i.c_p = 0
 * -------------------------------------------------------------------------------- */
enum { RULE_NONE = 0, RULE_PLANE, RULE_CONCAVE, RULE_CONVEX, RULE_CORNER, RULE_JUNCTION };

typedef struct {
  int type;
  int n[3]; /* plane: normal; edges: first plane normal; corner: (sx, sy, sz); junction: plane normal */
  int m[3]; /* edges: second plane normal */
  int d[3]; /* edges and junction: bulk normal of the edge */
} rule_t;

/* Split a diagonal lattice vector into its two axis components. */
static void split_diagonal(const int d[3], int a[3], int b[3]) {
  int first = 1;
  for (int i = 0; i < 3; ++i) a[i] = b[i] = 0;
  for (int i = 0; i < 3; ++i) {
    if (d[i] == 0) continue;
    if (first) { a[i] = d[i]; first = 0; }
    else b[i] = d[i];
  }
}

static int decode_rule(int code, rule_t* r) {
  memset(r, 0, sizeof(*r));
  int ac = code < 0 ? -code : code;
  if (code >= 1 && code <= 6) {
    r->type = RULE_PLANE;
    for (int i = 0; i < 3; ++i) r->n[i] = CV[code - 1][i];
  } else if (ac >= 7 && ac <= 18) {
    r->type = code > 0 ? RULE_CONCAVE : RULE_CONVEX;
    for (int i = 0; i < 3; ++i) r->d[i] = CV[ac - 1][i];
    split_diagonal(r->d, r->n, r->m);
  } else if (code >= 19 && code <= 26) {
    int b = code - 19;
    r->type = RULE_CORNER;
    r->n[0] = (b & 1) ? -1 : 1;
    r->n[1] = (b & 2) ? -1 : 1;
    r->n[2] = (b & 4) ? -1 : 1;
  } else if (code >= 27 && code <= 50) {
    int p = (code - 27) / 4, j = (code - 27) % 4, seen = 0;
    r->type = RULE_JUNCTION;
    for (int i = 0; i < 3; ++i) r->n[i] = CV[p][i];
    for (int k = 6; k < 18; ++k) {
      if (dot_ci(k, r->n) != 0) continue;
      if (seen++ == j) {
        for (int i = 0; i < 3; ++i) r->d[i] = CV[k][i];
        break;
      }
    }
  } else {
    return ORC_ERR_ARG;
  }
  return ORC_OK;
}

static int same_vector(int k, const int v[3]) { return CV[k][0] == v[0] && CV[k][1] == v[1] && CV[k][2] == v[2]; }

/* Populations the rule overwrites (its unknowns). */
static int rule_unknown(const rule_t* r, int k) {
  switch (r->type) {
    case RULE_PLANE: return dot_ci(k, r->n) > 0;
    case RULE_CONCAVE: return dot_ci(k, r->n) > 0 || dot_ci(k, r->m) > 0;
    case RULE_CONVEX: return same_vector(k, r->d);
    case RULE_CORNER:
      return CV[k][0] * r->n[0] > 0 || CV[k][1] * r->n[1] > 0 || CV[k][2] * r->n[2] > 0;
    case RULE_JUNCTION: return dot_ci(k, r->n) > 0 || same_vector(k, r->d);
    default: return 0;
  }
}

/* Convex edge (eq. edge2, reading R9): the population coming from the solid side is
 * bounced back; then N_i = 1/4 (c_i.e) sum_j f_j (c_j.e), e = n1 x n2, is subtracted
 * from every population travelling into the bulk (c_i.d > 0). */
static void close_convex_edge(double* f, const rule_t* r) {
  int e[3] = {r->n[1] * r->m[2] - r->n[2] * r->m[1], r->n[2] * r->m[0] - r->n[0] * r->m[2],
              r->n[0] * r->m[1] - r->n[1] * r->m[0]};
  for (int k = 0; k < Q; ++k)
    if (same_vector(k, r->d)) f[k] = f[opposite(k)];
  double P = 0.0;
  for (int j = 0; j < Q; ++j) P += f[j] * dot_ci(j, e);
  for (int k = 0; k < Q; ++k)
    if (dot_ci(k, r->d) > 0) f[k] -= 0.25 * dot_ci(k, e) * P;
}

/* Junction of a convex edge with a perpendicular plane (reading R10): bounce-back of
 * the populations coming from outside (through the plane or from the edge's solid
 * side), rest population = 12/36 of the node density. */
static void close_junction(double* f, const rule_t* r) {
  for (int k = 0; k < Q; ++k)
    if (rule_unknown(r, k)) f[k] = f[opposite(k)];
  double s = 0.0;
  for (int k = 0; k < Q - 1; ++k) s += f[k];
  F(19) = 0.5 * s;
}

/* Applies the rule of a node code (all velocities zero: no-slip walls). */
static int close_rule(int code, double* f, int form) {
  rule_t r;
  if (decode_rule(code, &r)) return ORC_ERR_ARG;
  static const double zero[3] = {0.0, 0.0, 0.0};
  switch (r.type) {
    case RULE_PLANE: close_face_form(code - 1, form, f, zero, -1.0); break;
    case RULE_CONCAVE: close_edge_normals(f, r.n, r.m, -1.0); break;
    case RULE_CONVEX: close_convex_edge(f, &r); break;
    case RULE_CORNER: {
      int n1[3] = {r.n[0], 0, 0}, n2[3] = {0, r.n[1], 0}, n3[3] = {0, 0, r.n[2]};
      close_corner_normals(f, n1, n2, n3, -1.0);
      break;
    }
    case RULE_JUNCTION: close_junction(f, &r); break;
    default: return ORC_ERR_ARG;
  }
  return ORC_OK;
}

int orc_close_rule(int code, double* f) { return close_rule(code, f, 0); }

/* unknown[k] = 1 where the rule of `code` overwrites population k. */
int orc_rule_unknowns(int code, int* unknown) {
  rule_t r;
  if (decode_rule(code, &r)) return ORC_ERR_ARG;
  for (int k = 0; k < Q; ++k) unknown[k] = rule_unknown(&r, k);
  return ORC_OK;
}

/* ----------------------------------------------------------------------------------
 * Lattice: streaming, classification, one time step.
 * -------------------------------------------------------------------------------- */
typedef struct {
  int nx, ny, nz;
  int kind[6];            /* 0 periodic, 1 velocity, 2 pressure */
  const double* utab[6];  /* [n2][n1][3] per velocity or pressure face (pressure: the
                             tangential velocity; the normal component is ignored) */
  const double* ptab[6];  /* [n2][n1] prescribed density per pressure face */
  const unsigned char* solid; /* optional [nz][ny][nx]: nonzero marks a solid node */
  const signed char* code;    /* optional [nz][ny][nx]: boundary rule of the node (0: none) */
  double force[3];            /* body force (eq. gravity) */
  int forced;                 /* force != 0 */
  double tau;
} lattice_t;

static int axis_dim(const lattice_t* L, int a) { return a == 0 ? L->nx : (a == 1 ? L->ny : L->nz); }
static int axis_periodic(const lattice_t* L, int a) { return L->kind[2 * a] == 0; }

static int lattice_check(const lattice_t* L) {
  if (L->nx < 1 || L->ny < 1 || L->nz < 1) return ORC_ERR_ARG;
  int pressure_axes = 0;
  for (int a = 0; a < 3; ++a) {
    for (int s = 0; s < 2; ++s) {
      int k = L->kind[2 * a + s];
      if (k < 0 || k > 2) return ORC_ERR_ARG;
      if (k != 0 && !L->utab[2 * a + s]) return ORC_ERR_ARG;
      if (k == 2 && !L->ptab[2 * a + s]) return ORC_ERR_ARG;
    }
    /* periodic faces come in pairs */
    if ((L->kind[2 * a] == 0) != (L->kind[2 * a + 1] == 0)) return ORC_ERR_ARG;
    if (L->kind[2 * a] != 0 && axis_dim(L, a) < 3) return ORC_ERR_ARG;
    if (L->kind[2 * a] == 2 || L->kind[2 * a + 1] == 2) ++pressure_axes;
  }
  /* an edge or corner borders at most one pressure plane */
  return pressure_axes <= 1 ? ORC_OK : ORC_ERR_ARG;
}

/* Linear index of the node that population k at (x,y,z) is pulled from, i.e.
 * x - c_k (streaming step, with wrap-around on periodic axes), or -1 when that node
 * lies outside the domain (the population is unknown after streaming). */
static int64_t pull_source(const lattice_t* L, int x, int y, int z, int k) {
  int p[3] = {x - CV[k][0], y - CV[k][1], z - CV[k][2]};
  for (int a = 0; a < 3; ++a) {
    int n = axis_dim(L, a);
    if (p[a] < 0 || p[a] >= n) {
      if (!axis_periodic(L, a)) return -1;
      p[a] = ((p[a] % n) + n) % n;
    }
  }
  return ((int64_t)p[2] * L->ny + p[1]) * L->nx + p[0];
}

/* Table position of node (x,y,z) on face `face` (tangential axes in increasing order). */
static int64_t face_index(const lattice_t* L, int face, int x, int y, int z) {
  int c[3] = {x, y, z};
  int a = face / 2, t1 = (a == 0) ? 1 : 0, t2 = (a == 2) ? 1 : 2;
  return (int64_t)c[t2] * axis_dim(L, t1) + c[t1];
}

/* Boundary closure and collision of one node whose streamed populations are in f
 * (NaN marks an unknown population). */
static int update_node(const lattice_t* L, int x, int y, int z, double* f, int form) {
  int c[3] = {x, y, z};
  int code = L->code ? L->code[((int64_t)z * L->ny + y) * L->nx + x] : 0;
  if (code != 0) {
    if (close_rule(code, f, form)) return ORC_ERR_ARG;
    for (int k = 0; k < Q; ++k)
      if (isnan(f[k])) return ORC_ERR_UNFILLED;
    if (L->forced) orc_collide_force(f, L->tau, L->force);
    else orc_collide(f, L->tau);
    return ORC_OK;
  }
  int faces[3], nf = 0;
  double rho_p = -1.0; /* density of a bordering pressure plane, if any */
  for (int a = 0; a < 3; ++a) {
    if (axis_periodic(L, a)) continue;
    int fc = -1;
    if (c[a] == 0) fc = 2 * a;
    else if (c[a] == axis_dim(L, a) - 1) fc = 2 * a + 1;
    if (fc < 0) continue;
    faces[nf++] = fc;
    if (L->kind[fc] == 2) rho_p = L->ptab[fc][face_index(L, fc, x, y, z)];
  }
  if (nf == 1) {
    const double* u = L->utab[faces[0]] + 3 * face_index(L, faces[0], x, y, z);
    if (L->kind[faces[0]] == 2) orc_close_face_pressure(faces[0], form, f, rho_p, u, NULL);
    else close_face_form(faces[0], form, f, u, -1.0);
  } else if (nf == 2) {
    int n1[3], n2[3];
    face_normal(faces[0], n1);
    face_normal(faces[1], n2);
    close_edge_normals(f, n1, n2, rho_p);
  } else if (nf == 3) {
    int n1[3], n2[3], n3[3];
    face_normal(faces[0], n1);
    face_normal(faces[1], n2);
    face_normal(faces[2], n3);
    close_corner_normals(f, n1, n2, n3, rho_p);
  }
  for (int k = 0; k < Q; ++k)
    if (isnan(f[k])) return ORC_ERR_UNFILLED;
  if (L->forced) orc_collide_force(f, L->tau, L->force);
  else orc_collide(f, L->tau);
  return ORC_OK;
}

static int make_lattice(lattice_t* L, int nx, int ny, int nz, const int* kind, const double* const* utab,
                        const double* const* ptab, double tau) {
  L->nx = nx; L->ny = ny; L->nz = nz; L->tau = tau;
  L->solid = NULL;
  L->code = NULL;
  L->force[0] = L->force[1] = L->force[2] = 0.0;
  L->forced = 0;
  for (int i = 0; i < 6; ++i) {
    L->kind[i] = kind[i];
    L->utab[i] = utab ? utab[i] : NULL;
    L->ptab[i] = ptab ? ptab[i] : NULL;
  }
  return lattice_check(L);
}

/* Flat index (population * N + node) that population k of node (x,y,z) takes its
 * streamed value from, or -1 when unknown. Pull streaming (Sec. "Simulation method"):
 * population k of node x - c_k. Next to a solid node the mid-grid bounce-back of
 * Sec. "Boundary conditions" applies instead: the population that node x sent towards
 * the solid node returns reversed, i.e. population -k of node x itself. */
static int64_t gather_source(const lattice_t* L, int x, int y, int z, int k) {
  int64_t N = (int64_t)L->nx * L->ny * L->nz;
  int64_t node = ((int64_t)z * L->ny + y) * L->nx + x;
  int64_t s = pull_source(L, x, y, z, k);
  if (s < 0) return -1;
  if (L->solid && L->solid[s]) {
    /* a node with an on-site rule overwrites this population (checked beforehand) */
    if (L->code && L->code[node] != 0) return -1;
    return (int64_t)opposite(k) * N + node;
  }
  return (int64_t)k * N + s;
}

/* Geometry check: a node with a rule is fluid, its code is valid, and every population
 * it cannot stream (source solid or outside a walled axis) is one the rule overwrites.
 * Returns the first offending node + 1 in *bad (0 if none). */
static int geometry_check(const lattice_t* L, int64_t* bad) {
  *bad = 0;
  if (!L->code) return ORC_OK;
  for (int z = 0; z < L->nz; ++z)
    for (int y = 0; y < L->ny; ++y)
      for (int x = 0; x < L->nx; ++x) {
        int64_t node = ((int64_t)z * L->ny + y) * L->nx + x;
        int code = L->code[node];
        if (code == 0) continue;
        rule_t r;
        int ok = !decode_rule(code, &r) && !(L->solid && L->solid[node]);
        for (int k = 0; ok && k < Q; ++k) {
          int64_t s = pull_source(L, x, y, z, k);
          int blocked = s < 0 || (L->solid && L->solid[s]);
          if (blocked && !rule_unknown(&r, k)) ok = 0;
        }
        if (!ok) {
          *bad = node + 1;
          return ORC_ERR_ARG;
        }
      }
  return ORC_OK;
}

int orc_check_geometry(int nx, int ny, int nz, const int* kind, const unsigned char* solid, const signed char* code,
                       int64_t* bad) {
  lattice_t L;
  double dummy = 0.0;
  const double* none[6] = {&dummy, &dummy, &dummy, &dummy, &dummy, &dummy};
  int rc = make_lattice(&L, nx, ny, nz, kind, none, none, 1.0);
  if (rc) return rc;
  L.solid = solid;
  L.code = code;
  return geometry_check(&L, bad);
}

/* Pull streaming only: out[k][node] = in[k][node - c_k], NaN where unknown. */
int orc_stream(int nx, int ny, int nz, const int* kind, const double* fin, double* fout) {
  lattice_t L;
  double dummy = 0.0;
  const double* none[6] = {&dummy, &dummy, &dummy, &dummy, &dummy, &dummy}; /* tables unused by streaming */
  int rc = make_lattice(&L, nx, ny, nz, kind, none, none, 1.0);
  if (rc) return rc;
  int64_t N = (int64_t)nx * ny * nz;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int64_t node = ((int64_t)z * ny + y) * nx + x;
        for (int k = 0; k < Q; ++k) {
          int64_t s = pull_source(&L, x, y, z, k);
          fout[k * N + node] = (s < 0) ? NAN : fin[k * N + s];
        }
      }
  return ORC_OK;
}

/* One time step fin -> fout (streaming, closure, collision). */
/* One time step fin -> fout (streaming, closure, collision). Solid nodes (when a mask
 * is given) keep their populations unchanged. */
int orc_step_geom(int nx, int ny, int nz, const int* kind, const double* const* utab, const double* const* ptab,
                  const unsigned char* solid, const signed char* code, const double* force, double tau,
                  const double* fin, double* fout, int form) {
  lattice_t L;
  int rc = make_lattice(&L, nx, ny, nz, kind, utab, ptab, tau);
  if (rc) return rc;
  L.solid = solid;
  L.code = code;
  if (force) {
    for (int a = 0; a < 3; ++a) L.force[a] = force[a];
    L.forced = force[0] != 0.0 || force[1] != 0.0 || force[2] != 0.0;
  }
  int64_t bad;
  rc = geometry_check(&L, &bad);
  if (rc) return rc;
  int64_t N = (int64_t)nx * ny * nz;
  int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int z = 0; z < nz; ++z) {
    double f[Q];
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int64_t node = ((int64_t)z * ny + y) * nx + x;
        if (solid && solid[node]) {
          for (int k = 0; k < Q; ++k) fout[k * N + node] = fin[k * N + node];
          continue;
        }
        for (int k = 0; k < Q; ++k) {
          int64_t s = gather_source(&L, x, y, z, k);
          f[k] = (s < 0) ? NAN : fin[s];
        }
        err |= update_node(&L, x, y, z, f, form);
        for (int k = 0; k < Q; ++k) fout[k * N + node] = f[k];
      }
  }
  return err;
}

int orc_step(int nx, int ny, int nz, const int* kind, const double* const* utab, const double* const* ptab,
             double tau, const double* fin, double* fout, int form) {
  return orc_step_geom(nx, ny, nz, kind, utab, ptab, NULL, NULL, NULL, tau, fin, fout, form);
}

/* nsteps time steps; f holds the initial and the final state, work is scratch of the
 * same size. */
int orc_run_geom(int nx, int ny, int nz, const int* kind, const double* const* utab, const double* const* ptab,
                 const unsigned char* solid, const signed char* code, const double* force, double tau, int nsteps,
                 double* f, double* work, int form) {
  int64_t n = (int64_t)Q * nx * ny * nz;
  double *a = f, *b = work;
  for (int s = 0; s < nsteps; ++s) {
    int rc = orc_step_geom(nx, ny, nz, kind, utab, ptab, solid, code, force, tau, a, b, form);
    if (rc) return rc;
    double* t = a; a = b; b = t;
  }
  if (a != f) memcpy(f, a, (size_t)n * sizeof(double));
  return ORC_OK;
}

int orc_run(int nx, int ny, int nz, const int* kind, const double* const* utab, const double* const* ptab,
            double tau, int nsteps, double* f, double* work, int form) {
  return orc_run_geom(nx, ny, nz, kind, utab, ptab, NULL, NULL, NULL, tau, nsteps, f, work, form);
}

/* f = f_eq(rho0, 0) on every node (the initial, post-collision state). */
void orc_init_equilibrium(int nx, int ny, int nz, double rho0, double* f) {
  int64_t N = (int64_t)nx * ny * nz;
  double v0[3] = {0, 0, 0}, feq[Q];
  orc_feq(rho0, v0, feq);
  for (int k = 0; k < Q; ++k)
    for (int64_t i = 0; i < N; ++i) f[k * N + i] = feq[k];
}

/* Density [nz][ny][nx] and velocity [3][nz][ny][nx] of a stored state. */
void orc_macros(int nx, int ny, int nz, const double* f, double* rho, double* u) {
  int64_t N = (int64_t)nx * ny * nz;
  for (int64_t i = 0; i < N; ++i) {
    double g[Q], m[4];
    for (int k = 0; k < Q; ++k) g[k] = f[k * N + i];
    orc_moments(g, m);
    rho[i] = m[0];
    for (int a = 0; a < 3; ++a) u[a * N + i] = m[a + 1];
  }
}

/* Reductions in node order: out = {sum rho, sum |u - u_prev|^2, sum |u|^2,
 * number of nodes with a non-finite or non-positive density or velocity}.
 * u_prev may be NULL (taken as zero). */
void orc_reduce(int nx, int ny, int nz, const double* f, const double* u_prev, double* out) {
  int64_t N = (int64_t)nx * ny * nz;
  double mass = 0, du2 = 0, u2 = 0, bad = 0;
  for (int64_t i = 0; i < N; ++i) {
    double g[Q], m[4];
    for (int k = 0; k < Q; ++k) g[k] = f[k * N + i];
    orc_moments(g, m);
    int ok = isfinite(m[0]) && m[0] > 0;
    for (int a = 0; a < 3; ++a) {
      double up = u_prev ? u_prev[a * N + i] : 0.0;
      du2 += (m[a + 1] - up) * (m[a + 1] - up);
      u2 += m[a + 1] * m[a + 1];
      ok = ok && isfinite(m[a + 1]);
    }
    mass += m[0];
    bad += ok ? 0 : 1;
  }
  out[0] = mass; out[1] = du2; out[2] = u2; out[3] = bad;
}

/* Pull sources of a list of nodes: src[i*19 + k] = k*N + (node - c_k) or -1. */
int orc_sources(int nx, int ny, int nz, const int* kind, int64_t n, const int64_t* nodes, int64_t* src) {
  lattice_t L;
  double dummy = 0.0;
  const double* none[6] = {&dummy, &dummy, &dummy, &dummy, &dummy, &dummy};
  int rc = make_lattice(&L, nx, ny, nz, kind, none, none, 1.0);
  if (rc) return rc;
  int64_t N = (int64_t)nx * ny * nz;
  for (int64_t i = 0; i < n; ++i) {
    int64_t node = nodes[i];
    if (node < 0 || node >= N) return ORC_ERR_ARG;
    int x = (int)(node % nx), y = (int)((node / nx) % ny), z = (int)(node / ((int64_t)nx * ny));
    for (int k = 0; k < Q; ++k) {
      int64_t s = pull_source(&L, x, y, z, k);
      src[i * Q + k] = (s < 0) ? -1 : (int64_t)k * N + s;
    }
  }
  return ORC_OK;
}

/* Closure and collision of listed nodes from their streamed populations
 * (g[i*19 + k], NaN where unknown); results in out[i*19 + k]. */
int orc_update_gathered(int nx, int ny, int nz, const int* kind, const double* const* utab,
                        const double* const* ptab, double tau, int64_t n, const int64_t* nodes,
                        const double* g, double* out, int form) {
  lattice_t L;
  int rc = make_lattice(&L, nx, ny, nz, kind, utab, ptab, tau);
  if (rc) return rc;
  int64_t N = (int64_t)nx * ny * nz;
  for (int64_t i = 0; i < n; ++i) {
    int64_t node = nodes[i];
    if (node < 0 || node >= N) return ORC_ERR_ARG;
    int x = (int)(node % nx), y = (int)((node / nx) % ny), z = (int)(node / ((int64_t)nx * ny));
    double f[Q];
    for (int k = 0; k < Q; ++k) f[k] = g[i * Q + k];
    rc = update_node(&L, x, y, z, f, form);
    if (rc) return rc;
    for (int k = 0; k < Q; ++k) out[i * Q + k] = f[k];
  }
  return ORC_OK;
}

/* Tables for inspection by the tests: c (19x3), w (19), opposite index (19). */
void orc_lattice(int* c, double* w, int* opp) {
  for (int k = 0; k < Q; ++k) {
    for (int a = 0; a < 3; ++a) c[3 * k + a] = CV[k][a];
    w[k] = WT[k];
    opp[k] = opposite(k);
  }
}

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
