/*
 * oracle.c -- plain, slow, float64 CPU reference of the time step of
 * Paquay & Kusters, "A method for molecular dynamics on curved surfaces":
 * RATTLE for particles held on an implicit surface g(x) = 0 (Algorithm 1)
 * combined with the Gronbech-Jensen/Farago Langevin form (Algorithm S1),
 * truncated-shifted Lennard-Jones pair forces (Eq. S1), harmonic bonds and
 * the repulsive Lennard-Jones wall (SI Section S3.2).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check of the package
 * entry point and the CPU-baseline leg of the benchmark may load this file's
 * library. It shares no code, header, table or constant with the CUDA path:
 * its structs, its Philox and its surface functions are written here from
 * their published definitions.
 *
 * Every loop follows the paper's order: for a step, first the position half
 * for all particles, then the forces, then the random force and the force
 * combination, then the momentum half (Algorithm S1). The Newton solves are
 * the 4x4 systems of Algorithm 1 with the Jacobians printed there, solved by
 * Gaussian elimination. Nothing is fused, blocked or reordered.
 *
 * Readings of points the paper leaves open (each is also stated where it is
 * used):
 *   R1  The Newton stopping test is |g|/|grad g| < eta and ||r_x||_inf < eta
 *       (g in any units becomes a length). A step smaller than 4 ulp of the
 *       iterate also ends the iteration (round-off floor).
 *   R2  The first combined force after a state is set is
 *       F = f(x) - gamma p + f_r (no noise average, no 1/(1+dt/2tau)).
 *   R3  The random force of step k is drawn from Philox4x32-10 with key
 *       (low 32 bits of seed, replica) and counter (particle, low 32 bits of
 *       k, high 32 bits of k, 0); the four words give three normals by
 *       Box-Muller: (w0, w1) -> (x, y), (w2, w3) -> z (cosine branch), with
 *       the uniform u(w) = ((w >> 9) + 1/2) 2^-23.
 *   R4  The torus is the connector form of SI S3.1 with its axis on z; the
 *       ellipsoid is sum (x_d/a_d)^2 - 1; the bump is z - A exp(-rho^2/2w^2)
 *       with rho taken with the minimum image in periodic x, y.
 *   R5  The bond potential carries no factor 1/2: V = k (r - r0)^2.
 *   R6  The wall V_w acts on unconstrained particles with r - R_w replaced by
 *       the distance to each of two planes z = wall_lo_z, z = wall_hi_z.
 *   R8  The bend angle theta of V_bend (SI S3.2) is the angle at the middle
 *       bead between x_i - x_j and x_k - x_j (pi for a straight chain, the
 *       rest angle theta0 = pi of the capsid model); the SI's arccos of
 *       (x_i - x_j).(x_j - x_k) / (...) would be 0 for a straight chain. It
 *       is evaluated as atan2(|u x w|, u.w), equal to the arccos and well
 *       conditioned near 0 and pi.
 *   R9  The thylakoid surface of SI S3.1 is assembled from its pieces as
 *       follows (p = (R_b, L_x, R_c, L_b), centre c, z periodic): a bridge
 *       cylinder of radius R_b along x through (c_y, c_z) for
 *       |x - c_x| <= L_b/2; at each end a connector (SI form, tube radius
 *       R = R_c) joining it tangentially to the face plane of a block at
 *       x = c_x -/+ (L_b/2 + R_c); each block a tube along z whose cross
 *       section is a square of side L_x + 2 R_c with its corners rounded by
 *       quarter cylinders of radius R_c (four planes L_x x L_z and four
 *       quarter cylinders, as the SI's area sum counts). The piece of a
 *       particle is chosen from the position where its half step starts:
 *       between the block faces and within R_b + R_c of the bridge axis the
 *       bridge or the nearer connector (by x against the bridge ends);
 *       otherwise the block's rounded square: a corner cylinder where the
 *       point lies beyond the inner square in both x and y, else the plane
 *       of the side it lies beyond (the nearest side when inside), except
 *       that the face plane's hole (within R_b + R_c of the axis) belongs to
 *       the connector. The pieces meet with continuous tangent planes.
 *   R7  The linearly smoothed Lennard-Jones potential is printed with
 *       "+ (r - r_c) phi'(r_c)", whose force does not vanish at r_c (it
 *       doubles the jump); the text states that energy and force are both
 *       continuous at r_c, which holds for "- (r - r_c) phi'(r_c)", the form
 *       used here.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXT 8

/* ------------------------------------------------------------------------ */
/* Public structs (mirrored by the ctypes wrapper in __init__.py).          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t kind; /* 0 none, 1 plane, 2 sphere, 3 ellipsoid, 4 torus,
                   5 gaussian bump, 6 cylinder, 7 unconstrained 2D plane
                   z = c[2] (no z updates; the baseline of Section 3.1's
                   performance comparison), 8 thylakoid composite (SI S3.1,
                   reading R9) */
  int32_t pad;
  double c[3];
  double p[4];
} orc_surface;

typedef struct {
  double dt, kT, gamma, tol;
  int32_t max_newton, ntypes, beads_per_mol, exclude_intramol;
  double mass[ORC_MAXT];
  double eps[ORC_MAXT][ORC_MAXT];
  double sigma[ORC_MAXT][ORC_MAXT];
  double rcut[ORC_MAXT][ORC_MAXT];
  double box_lo[3], box_hi[3];
  int32_t periodic[3];
  int32_t wall_enable;
  double bond_k, bond_r0;
  double wall_lo_z, wall_hi_z, wall_eps, wall_sigma;
  uint64_t seed;
  uint32_t replica;
  int32_t force_mode; /* 0: brute force up to 4000 particles, else cells;
                         1: brute force; 2: cell list */
  int32_t pair_form;  /* 0: truncated and shifted (Eq. S1); 1: linearly
                         smoothed (V*_LJ of the energy-conservation study) */
  /* capsid-model terms (SI S3.2) */
  double angle_k, angle_theta0;
  int32_t bond_r0_mix; /* 1: bond rest length 2^(1/6) sigma[ti][tj] / 2 */
  int32_t wall_kind;   /* 0: planes z = wall_lo_z, wall_hi_z; 1: sphere */
  double wall_radius;
  double wall_center[3];
} orc_params;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64 multiplications with  */
/* the published multipliers, the key bumped by the published Weyl words.   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Reading R3: three standard normals of particle `pid` at step `step`. */
void orc_gauss3(uint64_t seed, uint32_t replica, uint32_t pid, uint64_t step,
                double out[3]) {
  uint32_t ctr[4] = {pid, (uint32_t)(step & 0xffffffffu), (uint32_t)(step >> 32), 0u};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), replica};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  double u[4];
  for (int k = 0; k < 4; ++k) u[k] = ((double)(w[k] >> 9) + 0.5) * (1.0 / 8388608.0);
  const double two_pi = 6.283185307179586476925286766559;
  double r01 = sqrt(-2.0 * log(u[0]));
  double r23 = sqrt(-2.0 * log(u[2]));
  out[0] = r01 * cos(two_pi * u[1]);
  out[1] = r01 * sin(two_pi * u[1]);
  out[2] = r23 * cos(two_pi * u[3]);
}

/* ------------------------------------------------------------------------ */
/* Geometry helpers                                                          */
/* ------------------------------------------------------------------------ */
static double box_len(const orc_params* P, int d) { return P->box_hi[d] - P->box_lo[d]; }

/* Minimum-image displacement along periodic axes. */
static void min_image(const orc_params* P, double d[3]) {
  for (int k = 0; k < 3; ++k)
    if (P->periodic[k]) {
      double L = box_len(P, k);
      d[k] -= L * floor(d[k] / L + 0.5);
    }
}

static double maxabs3(const double v[3]) {
  double m = fabs(v[0]);
  if (fabs(v[1]) > m) m = fabs(v[1]);
  if (fabs(v[2]) > m) m = fabs(v[2]);
  return m;
}

static double ulp_of(double v) {
  double a = fabs(v);
  return nextafter(a, INFINITY) - a;
}

/* g(x) and its unnormalised gradient n = dg/dx for each surface kind
 * (Eq. 1 text for the sphere, SI S3.1 for plane / cylinder / connector,
 * reading R4 for torus, ellipsoid and bump). */
/* Thylakoid pieces (reading R9). type: 0 plane normal to x, 1 plane normal
 * to y (g = s (x_d - c)), 2 cylinder along z about (c0, c1) with radius rad,
 * 3 the bridge (cylinder along x), 4 a connector whose circle centre sits at
 * x = c0. */
typedef struct {
  int type;
  double s, c0, c1, rad;
} thyl_piece;

static double thyl_dz(const orc_surface* S, const orc_params* P, double z) {
  double d[3] = {0.0, 0.0, z - S->c[2]};
  min_image(P, d);
  return d[2];
}

static thyl_piece thyl_select(const orc_surface* S, const orc_params* P, const double x[3]) {
  double Rb = S->p[0], Lx = S->p[1], Rc = S->p[2], Lb = S->p[3];
  double xc = S->c[0], yc = S->c[1];
  double x0L = xc - 0.5 * Lb, x0R = xc + 0.5 * Lb, xfL = x0L - Rc, xfR = x0R + Rc;
  double dy = x[1] - yc, dz = thyl_dz(S, P, x[2]);
  double r = sqrt(dy * dy + dz * dz), Rout = Rb + Rc;
  thyl_piece q = {0, 1.0, 0.0, 0.0, 0.0};
  if (x[0] > xfL && x[0] < xfR && r < Rout) {
    if (x[0] < x0L) { q.type = 4; q.c0 = x0L; }
    else if (x[0] > x0R) { q.type = 4; q.c0 = x0R; }
    else { q.type = 3; q.rad = Rb; }
    return q;
  }
  int left = x[0] <= xc;
  /* inner square of the block (centres of its corner cylinders) */
  double ixl = left ? xfL - Rc - Lx : xfR + Rc, ixh = ixl + Lx;
  double iyl = yc - 0.5 * Lx, iyh = yc + 0.5 * Lx;
  double ex = x[0] < ixl ? x[0] - ixl : (x[0] > ixh ? x[0] - ixh : 0.0);
  double ey = x[1] < iyl ? x[1] - iyl : (x[1] > iyh ? x[1] - iyh : 0.0);
  if (ex != 0.0 && ey != 0.0) {
    q.type = 2; q.c0 = ex < 0.0 ? ixl : ixh; q.c1 = ey < 0.0 ? iyl : iyh; q.rad = Rc;
    return q;
  }
  if (ex == 0.0 && ey == 0.0) { /* inside: the nearest side */
    double dxl = x[0] - (ixl - Rc), dxh = (ixh + Rc) - x[0], dyl = x[1] - (iyl - Rc), dyh = (iyh + Rc) - x[1];
    double mx = dxl < dxh ? dxl : dxh, my = dyl < dyh ? dyl : dyh;
    if (mx <= my) ex = dxl < dxh ? -1.0 : 1.0;
    else ey = dyl < dyh ? -1.0 : 1.0;
  }
  if (ex != 0.0) {
    int face = left ? ex > 0.0 : ex < 0.0; /* the side that faces the bridge */
    if (face && r < Rout) { q.type = 4; q.c0 = left ? x0L : x0R; return q; }
    q.type = 0; q.s = ex < 0.0 ? -1.0 : 1.0; q.c0 = ex < 0.0 ? ixl - Rc : ixh + Rc;
    return q;
  }
  q.type = 1; q.s = ey < 0.0 ? -1.0 : 1.0; q.c0 = ey < 0.0 ? iyl - Rc : iyh + Rc;
  return q;
}

static double thyl_eval(const orc_surface* S, const orc_params* P, const thyl_piece* q, const double x[3],
                        double n[3]) {
  double Rc = S->p[2], Rout = S->p[0] + Rc;
  double dy = x[1] - S->c[1], dz = thyl_dz(S, P, x[2]);
  switch (q->type) {
    case 0: n[0] = q->s; n[1] = 0.0; n[2] = 0.0; return q->s * (x[0] - q->c0);
    case 1: n[0] = 0.0; n[1] = q->s; n[2] = 0.0; return q->s * (x[1] - q->c0);
    case 2: {
      double a = x[0] - q->c0, b = x[1] - q->c1;
      n[0] = 2.0 * a; n[1] = 2.0 * b; n[2] = 0.0;
      return a * a + b * b - q->rad * q->rad;
    }
    case 3:
      n[0] = 0.0; n[1] = 2.0 * dy; n[2] = 2.0 * dz;
      return dy * dy + dz * dz - q->rad * q->rad;
    default: {
      double r = sqrt(dy * dy + dz * dz), a = x[0] - q->c0, t = r - Rout;
      double w = 2.0 * (1.0 - Rout / r);
      n[0] = 2.0 * a; n[1] = w * dy; n[2] = w * dz;
      return a * a + t * t - Rc * Rc;
    }
  }
}

/* g at x_eval on the piece selected at x_sel (the thylakoid; any other
 * surface is evaluated at x_eval). */
static double surface_g_from(const orc_surface* S, const orc_params* P, const double x_sel[3],
                             const double x_eval[3], double n[3]);

double orc_surface_g(const orc_surface* S, const orc_params* P, const double x[3],
                     double n[3]) {
  double d[3] = {x[0] - S->c[0], x[1] - S->c[1], x[2] - S->c[2]};
  switch (S->kind) {
    case 1: { /* plane */
      n[0] = S->p[0]; n[1] = S->p[1]; n[2] = S->p[2];
      return S->p[0] * d[0] + S->p[1] * d[1] + S->p[2] * d[2];
    }
    case 2: { /* sphere */
      double R = S->p[0];
      n[0] = 2.0 * d[0]; n[1] = 2.0 * d[1]; n[2] = 2.0 * d[2];
      return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - R * R;
    }
    case 3: { /* ellipsoid */
      double g = -1.0;
      for (int k = 0; k < 3; ++k) {
        double a2 = S->p[k] * S->p[k];
        g += d[k] * d[k] / a2;
        n[k] = 2.0 * d[k] / a2;
      }
      return g;
    }
    case 4: { /* torus: (rho - R)^2 + z^2 - r^2 */
      double R = S->p[0], r = S->p[1];
      double rho = sqrt(d[0] * d[0] + d[1] * d[1]);
      double t = rho - R;
      n[0] = 2.0 * t * d[0] / rho;
      n[1] = 2.0 * t * d[1] / rho;
      n[2] = 2.0 * d[2];
      return t * t + d[2] * d[2] - r * r;
    }
    case 5: { /* gaussian bump: z - A exp(-rho^2 / 2w^2) */
      double A = S->p[0], w = S->p[1];
      double dd[3] = {d[0], d[1], 0.0};
      min_image(P, dd);
      double rho2 = dd[0] * dd[0] + dd[1] * dd[1];
      double e = A * exp(-rho2 / (2.0 * w * w));
      n[0] = e * dd[0] / (w * w);
      n[1] = e * dd[1] / (w * w);
      n[2] = 1.0;
      return d[2] - e;
    }
    case 8: { /* thylakoid composite (reading R9): the piece at x */
      thyl_piece q = thyl_select(S, P, x);
      return thyl_eval(S, P, &q, x, n);
    }
    case 6: { /* cylinder, axis p[1] */
      double R = S->p[0];
      int ax = (int)S->p[1];
      double g = -R * R;
      for (int k = 0; k < 3; ++k) {
        if (k == ax) {
          n[k] = 0.0;
        } else {
          g += d[k] * d[k];
          n[k] = 2.0 * d[k];
        }
      }
      return g;
    }
    default:
      n[0] = n[1] = n[2] = 0.0;
      return 0.0;
  }
}

static double surface_g_from(const orc_surface* S, const orc_params* P, const double x_sel[3],
                             const double x_eval[3], double n[3]) {
  if (S->kind != 8) return orc_surface_g(S, P, x_eval, n);
  thyl_piece q = thyl_select(S, P, x_sel);
  return thyl_eval(S, P, &q, x_eval, n);
}

/* Solve the 4x4 system J d = r by Gaussian elimination with partial
 * pivoting (a library-style primitive: the step "J^{-1} r" of Algorithm 1).
 * Returns 0 on success, 1 if J is singular. */
static int solve4(double J[4][4], const double r[4], double d[4]) {
  double A[4][5];
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) A[i][j] = J[i][j];
    A[i][4] = r[i];
  }
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int i = col + 1; i < 4; ++i)
      if (fabs(A[i][col]) > fabs(A[piv][col])) piv = i;
    if (A[piv][col] == 0.0) return 1;
    if (piv != col)
      for (int j = 0; j < 5; ++j) {
        double t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t;
      }
    for (int i = col + 1; i < 4; ++i) {
      double f = A[i][col] / A[col][col];
      for (int j = col; j < 5; ++j) A[i][j] -= f * A[col][j];
    }
  }
  for (int i = 3; i >= 0; --i) {
    double s = A[i][4];
    for (int j = i + 1; j < 4; ++j) s -= A[i][j] * d[j];
    d[i] = s / A[i][i];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, position half, for one constrained particle.                */
/* Unknowns (x^{m+1}, lambda); start lambda = 0, x^{m+1} = x^m;             */
/*   p^{m+1/2} = p^m + dt/2 (f^m - lambda n^m)                              */
/*   r = (x^m - x^{m+1} + dt/m p^{m+1/2},  g(x^{m+1}))                      */
/*   J = [[-I, -dt^2/(2m) n^m], [n^{m+1 T}, 0]]                             */
/*   (x^{m+1}, lambda) <- (x^{m+1}, lambda) - J^{-1} r                       */
/* until ||r|| < eta (reading R1).                                          */
/* Returns 0 converged, 1 converged at the round-off floor, -1 not converged */
/* after max_it iterations, -2 singular Jacobian.                           */
/* ------------------------------------------------------------------------ */
int orc_position_half(const orc_surface* S, const orc_params* P, const double x[3],
                      const double p[3], const double f[3], double m,
                      double x_new[3], double p_half[3], double* lambda_out,
                      int32_t* iters_out) {
  const double dt = P->dt, eta = P->tol;
  double nm[3];
  orc_surface_g(S, P, x, nm);
  double lam = 0.0;
  double xn[3] = {x[0], x[1], x[2]};
  int status = -1;
  int it;
  for (it = 0; it <= P->max_newton; ++it) {
    double ph[3], rx[3], n1[3];
    for (int k = 0; k < 3; ++k) ph[k] = p[k] + 0.5 * dt * (f[k] - lam * nm[k]);
    for (int k = 0; k < 3; ++k) rx[k] = x[k] - xn[k] + dt / m * ph[k];
    double rg = surface_g_from(S, P, x, xn, n1); /* the piece of x^m (R9) */
    double gn = sqrt(n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2]);
    if (fabs(rg) / gn < eta && maxabs3(rx) < eta) {
      status = 0;
      break;
    }
    if (it == P->max_newton) break;
    double J[4][4] = {{-1.0, 0.0, 0.0, -dt * dt / (2.0 * m) * nm[0]},
                      {0.0, -1.0, 0.0, -dt * dt / (2.0 * m) * nm[1]},
                      {0.0, 0.0, -1.0, -dt * dt / (2.0 * m) * nm[2]},
                      {n1[0], n1[1], n1[2], 0.0}};
    double r[4] = {rx[0], rx[1], rx[2], rg}, d[4];
    if (solve4(J, r, d)) {
      status = -2;
      break;
    }
    for (int k = 0; k < 3; ++k) xn[k] -= d[k];
    lam -= d[3];
    double dxmax = maxabs3(d);
    if (dxmax <= 4.0 * ulp_of(maxabs3(xn))) {
      status = 1;
      break;
    }
  }
  for (int k = 0; k < 3; ++k) {
    p_half[k] = p[k] + 0.5 * dt * (f[k] - lam * nm[k]);
    x_new[k] = xn[k];
  }
  if (lambda_out) *lambda_out = lam;
  if (iters_out) *iters_out = it;
  return status;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, momentum half, for one constrained particle at x^{m+1}.     */
/* Unknowns (p^{m+1}, mu); start mu = 0, p^{m+1} = p^{m+1/2} + dt/2 f^{m+1}; */
/*   r = (p^{m+1/2} - p^{m+1} + dt/2 (f^{m+1} - mu n^{m+1}),                 */
/*        m^{-1} n^{m+1} . p^{m+1})                                          */
/*   J = [[-I, -dt/2 n^{m+1}], [m^{-1} n^{m+1 T}, 0]]                        */
/* until ||r|| < eta, the n.p row measured as |n.p|/(m |n|) (a velocity).   */
/* ------------------------------------------------------------------------ */
int orc_momentum_half(const orc_surface* S, const orc_params* P, const double x_new[3],
                      const double p_half[3], const double f_new[3], double m,
                      double p_new[3], double* mu_out, int32_t* iters_out) {
  const double dt = P->dt, eta = P->tol;
  double n1[3];
  orc_surface_g(S, P, x_new, n1);
  double gn = sqrt(n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2]);
  double mu = 0.0;
  double pn[3];
  for (int k = 0; k < 3; ++k) pn[k] = p_half[k] + 0.5 * dt * f_new[k];
  int status = -1;
  int it;
  for (it = 0; it <= P->max_newton; ++it) {
    double rp[3];
    for (int k = 0; k < 3; ++k)
      rp[k] = p_half[k] - pn[k] + 0.5 * dt * (f_new[k] - mu * n1[k]);
    double rnp = (n1[0] * pn[0] + n1[1] * pn[1] + n1[2] * pn[2]) / m;
    if (maxabs3(rp) < eta && fabs(rnp) / gn < eta) {
      status = 0;
      break;
    }
    if (it == P->max_newton) break;
    double J[4][4] = {{-1.0, 0.0, 0.0, -0.5 * dt * n1[0]},
                      {0.0, -1.0, 0.0, -0.5 * dt * n1[1]},
                      {0.0, 0.0, -1.0, -0.5 * dt * n1[2]},
                      {n1[0] / m, n1[1] / m, n1[2] / m, 0.0}};
    double r[4] = {rp[0], rp[1], rp[2], rnp}, d[4];
    if (solve4(J, r, d)) {
      status = -2;
      break;
    }
    for (int k = 0; k < 3; ++k) pn[k] -= d[k];
    mu -= d[3];
    if (maxabs3(d) <= 4.0 * ulp_of(maxabs3(pn))) {
      status = 1;
      break;
    }
  }
  for (int k = 0; k < 3; ++k) p_new[k] = pn[k];
  if (mu_out) *mu_out = mu;
  if (iters_out) *iters_out = it;
  return status;
}

/* ------------------------------------------------------------------------ */
/* Forces: f = -grad V                                                       */
/* ------------------------------------------------------------------------ */
/* Lennard-Jones pair term at displacement d = x_i - x_j, with
 * phi(r) = 4 eps [(s/r)^12 - (s/r)^6]:
 *   pair_form 0, truncated and shifted (Eq. S1):  V = phi(r) - phi(r_c);
 *   pair_form 1, linearly smoothed (energy-conservation study of the SI):
 *                V = phi(r) - phi(r_c) - (r - r_c) phi'(r_c)   (reading R7),
 * both 0 for r >= r_c. Adds the force -dV/dr d/r on i to fi and returns V. */
static double lj_pair(const orc_params* P, int ti, int tj, const double d[3],
                      double fi[3]) {
  double rc = P->rcut[ti][tj];
  if (rc <= 0.0) return 0.0;
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (r2 >= rc * rc) return 0.0;
  double eps = P->eps[ti][tj], sig = P->sigma[ti][tj];
  double r = sqrt(r2);
  double sr6 = pow(sig / r, 6.0);
  double sr12 = sr6 * sr6;
  double src6 = pow(sig / rc, 6.0);
  double phi = 4.0 * eps * (sr12 - sr6);
  double phic = 4.0 * eps * (src6 * src6 - src6);
  /* -dphi/dr = 24 eps (2 (s/r)^12 - (s/r)^6) / r; along d/r */
  double fr_over_r = 24.0 * eps * (2.0 * sr12 - sr6) / r2;
  double v = phi - phic;
  if (P->pair_form == 1) {
    /* phi'(r_c) = -24 eps (2 (s/r_c)^12 - (s/r_c)^6) / r_c; the linear term
       adds +phi'(r_c) to -dV/dr, so the force vanishes at r_c */
    double dphic = -24.0 * eps * (2.0 * src6 * src6 - src6) / rc;
    v -= (r - rc) * dphic;
    fr_over_r += dphic / r;
  }
  for (int k = 0; k < 3; ++k) fi[k] += fr_over_r * d[k];
  return v;
}

static int same_molecule(const orc_params* P, const int32_t* mol, int64_t i, int64_t j) {
  if (!P->exclude_intramol) return 0;
  return mol[i] == mol[j];
}

/* All pairs i < j (minimum image). f and u are overwritten. */
void orc_pair_forces_brute(const orc_params* P, int64_t n, const double* x,
                           const int32_t* type, const int32_t* mol, double* f,
                           double* u) {
  memset(f, 0, sizeof(double) * 3 * (size_t)n);
  if (u) memset(u, 0, sizeof(double) * (size_t)n);
  int any = 0;
  for (int a = 0; a < P->ntypes; ++a)
    for (int b = 0; b < P->ntypes; ++b)
      if (P->rcut[a][b] > 0.0) any = 1;
  if (!any) return; /* no pair term at all */
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = i + 1; j < n; ++j) {
      if (same_molecule(P, mol, i, j)) continue;
      double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1],
                     x[3 * i + 2] - x[3 * j + 2]};
      min_image(P, d);
      double fi[3] = {0, 0, 0};
      double v = lj_pair(P, type[i], type[j], d, fi);
      for (int k = 0; k < 3; ++k) {
        f[3 * i + k] += fi[k];
        f[3 * j + k] -= fi[k];
      }
      if (u) {
        u[i] += 0.5 * v;
        u[j] += 0.5 * v;
      }
    }
  }
}

/* A simple cell list: every particle is binned into a grid of cells no
 * smaller than the largest cutoff, the (cell, particle) pairs are sorted,
 * and each particle visits the distinct cells among its 27 neighbours (found
 * by binary search). Each pair is evaluated from both sides. */
typedef struct {
  int64_t key;
  int64_t idx;
} orc_kv;

static int kv_cmp(const void* a, const void* b) {
  const orc_kv* A = (const orc_kv*)a;
  const orc_kv* B = (const orc_kv*)b;
  if (A->key != B->key) return A->key < B->key ? -1 : 1;
  return A->idx < B->idx ? -1 : (A->idx > B->idx ? 1 : 0);
}

static int64_t kv_lower(const orc_kv* a, int64_t n, int64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (a[mid].key < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

int orc_pair_forces_cells(const orc_params* P, int64_t n, const double* x,
                          const int32_t* type, const int32_t* mol, double* f,
                          double* u) {
  memset(f, 0, sizeof(double) * 3 * (size_t)n);
  if (u) memset(u, 0, sizeof(double) * (size_t)n);
  if (n == 0) return 0;
  double rc = 0.0;
  for (int a = 0; a < P->ntypes; ++a)
    for (int b = 0; b < P->ntypes; ++b)
      if (P->rcut[a][b] > rc) rc = P->rcut[a][b];
  if (rc <= 0.0) return 0;
  double lo[3], hi[3], cs[3];
  int64_t nc[3];
  for (int k = 0; k < 3; ++k) {
    if (P->periodic[k]) {
      lo[k] = P->box_lo[k];
      hi[k] = P->box_hi[k];
    } else {
      lo[k] = hi[k] = x[k];
      for (int64_t i = 1; i < n; ++i) {
        if (x[3 * i + k] < lo[k]) lo[k] = x[3 * i + k];
        if (x[3 * i + k] > hi[k]) hi[k] = x[3 * i + k];
      }
      hi[k] += 1e-9 * (1.0 + fabs(hi[k]));
    }
    double span = hi[k] - lo[k];
    nc[k] = (int64_t)floor(span / rc);
    if (nc[k] < 1) nc[k] = 1;
    cs[k] = span / (double)nc[k];
    if (cs[k] <= 0.0) cs[k] = rc;
  }
  orc_kv* kv = (orc_kv*)malloc(sizeof(orc_kv) * (size_t)n);
  int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)n);
  if (!kv || !cell) {
    free(kv);
    free(cell);
    return -1;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c[3];
    for (int k = 0; k < 3; ++k) {
      double xk = x[3 * i + k];
      if (P->periodic[k]) {
        double L = hi[k] - lo[k];
        xk -= L * floor((xk - lo[k]) / L);
      }
      int64_t ck = (int64_t)floor((xk - lo[k]) / cs[k]);
      if (ck < 0) ck = 0;
      if (ck > nc[k] - 1) ck = nc[k] - 1;
      c[k] = ck;
      cell[3 * i + k] = ck;
    }
    kv[i].key = c[0] + nc[0] * (c[1] + nc[1] * c[2]);
    kv[i].idx = i;
  }
  qsort(kv, (size_t)n, sizeof(orc_kv), kv_cmp);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    int64_t seen[27];
    int nseen = 0;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int64_t c[3] = {cell[3 * i] + dx, cell[3 * i + 1] + dy, cell[3 * i + 2] + dz};
          int ok = 1;
          for (int k = 0; k < 3; ++k) {
            if (c[k] < 0 || c[k] >= nc[k]) {
              if (P->periodic[k]) c[k] = (c[k] + nc[k]) % nc[k];
              else ok = 0;
            }
          }
          if (!ok) continue;
          int64_t key = c[0] + nc[0] * (c[1] + nc[1] * c[2]);
          int dup = 0;
          for (int s = 0; s < nseen; ++s)
            if (seen[s] == key) dup = 1;
          if (dup) continue;
          seen[nseen++] = key;
          for (int64_t q = kv_lower(kv, n, key); q < n && kv[q].key == key; ++q) {
            int64_t j = kv[q].idx;
            if (j == i || same_molecule(P, mol, i, j)) continue;
            double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1],
                           x[3 * i + 2] - x[3 * j + 2]};
            min_image(P, d);
            double v = lj_pair(P, type[i], type[j], d, &f[3 * i]);
            if (u) u[i] += 0.5 * v;
          }
        }
  }
  free(kv);
  free(cell);
  return 0;
}

/* Harmonic bonds along each molecule's chain (reading R5) and the wall of
 * reading R6; both add to f and u. Returns 1 if a free particle sits on or
 * behind a wall plane. */
/* Bend angle of three beads (SI S3.2, reading R8): u = x_a - x_m,
 * w = x_b - x_m, theta = atan2(|u x w|, u.w), V = k (theta - theta0)^2.
 * With c = cos(theta), s = sin(theta), dV = dV/dtheta = 2 k (theta - theta0):
 *   F_a = (dV / s) (w / (|u| |w|) - c u / |u|^2),
 *   F_b = (dV / s) (u / (|u| |w|) - c w / |w|^2),   F_m = -(F_a + F_b)
 * (F = -dV/dx with dtheta/dc = -1/s). At s = 0 the bracket is zero. */
static double angle_term(const orc_params* P, const double xa[3], const double xm[3], const double xb[3],
                         double fa[3], double fm[3], double fb[3]) {
  double u[3] = {xa[0] - xm[0], xa[1] - xm[1], xa[2] - xm[2]};
  double w[3] = {xb[0] - xm[0], xb[1] - xm[1], xb[2] - xm[2]};
  min_image(P, u);
  min_image(P, w);
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double uw = u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
  double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
  double sn = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  double theta = atan2(sn, uw);
  double norm = sqrt(uu * ww);
  double c = uw / norm, sth = sn / norm;
  double dV = 2.0 * P->angle_k * (theta - P->angle_theta0);
  double ratio = sth > 0.0 ? dV / sth : 0.0;
  for (int k = 0; k < 3; ++k) {
    fa[k] = ratio * (w[k] / norm - c * u[k] / uu);
    fb[k] = ratio * (u[k] / norm - c * w[k] / ww);
    fm[k] = -(fa[k] + fb[k]);
  }
  return P->angle_k * (theta - P->angle_theta0) * (theta - P->angle_theta0);
}

static double bond_r0_of(const orc_params* P, const int32_t* type, int64_t i, int64_t j) {
  if (!P->bond_r0_mix) return P->bond_r0;
  int ti = type ? type[i] : 0, tj = type ? type[j] : 0;
  return pow(2.0, 1.0 / 6.0) * P->sigma[ti][tj] / 2.0;
}

/* Wall V_w of SI S3.2 on one unconstrained particle: planes z = wall_lo_z and
 * z = wall_hi_z (reading R6), or the sphere of radius wall_radius about
 * wall_center (r - R_w with r the distance from the centre, pushing outward).
 * Adds the force to f and returns the energy; sets *bad behind a wall. */
static double wall_term(const orc_params* P, const double xi[3], double f[3], double* scale, int* bad) {
  double sw = P->wall_sigma, ew = P->wall_eps, v = 0.0;
  double rcw = pow(2.0, 1.0 / 6.0) * sw;
  if (P->wall_kind == 1) {
    double d[3] = {xi[0] - P->wall_center[0], xi[1] - P->wall_center[1], xi[2] - P->wall_center[2]};
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double h = r - P->wall_radius;
    if (h <= 0.0) {
      if (bad) *bad = 1;
      return 0.0;
    }
    if (h >= rcw) return 0.0;
    double s6 = pow(sw / h, 6.0);
    double fr = 24.0 * ew * (2.0 * s6 * s6 - s6) / h;
    for (int k = 0; k < 3; ++k) f[k] += fr * d[k] / r;
    if (scale) *scale += fabs(fr);
    return 4.0 * ew * (s6 * s6 - s6 + 0.25);
  }
  double dist[2] = {xi[2] - P->wall_lo_z, P->wall_hi_z - xi[2]};
  double sign[2] = {+1.0, -1.0};
  for (int w = 0; w < 2; ++w) {
    double r = dist[w];
    if (r <= 0.0) {
      if (bad) *bad = 1;
      continue;
    }
    if (r >= rcw) continue;
    double s6 = pow(sw / r, 6.0);
    double fr = 24.0 * ew * (2.0 * s6 * s6 - s6) / r;
    f[2] += sign[w] * fr;
    if (scale) *scale += fabs(fr);
    v += 4.0 * ew * (s6 * s6 - s6 + 0.25);
  }
  return v;
}

/* Bonded and wall terms acting on particle i (SI S3.2): the bonds to its
 * chain neighbours, every bend angle of three consecutive beads containing
 * i, and the wall (unconstrained particles). Adds the force on i to f and
 * returns i's share of the energy (half of each bond, a third of each angle,
 * all of its wall term); adds each term's force magnitude on i to *scale. */
static double bonded_on(const orc_params* P, int64_t n, const double* x, const int32_t* type,
                        const uint8_t* con, int64_t i, double f[3], double* scale, int* bad) {
  double ui = 0.0;
  int64_t B = P->beads_per_mol;
  if (B > 1) {
    for (int side = 0; side < 2; ++side) {
      int64_t j = side == 0 ? i - 1 : i + 1;
      if (side == 0 && (i % B) == 0) continue;
      if (side == 1 && ((i % B) == B - 1 || j >= n)) continue;
      double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
      min_image(P, d);
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double dr = r - bond_r0_of(P, type, i, j);
      for (int k = 0; k < 3; ++k) f[k] += -2.0 * P->bond_k * dr / r * d[k];
      if (scale) *scale += fabs(2.0 * P->bond_k * dr);
      ui += 0.5 * P->bond_k * dr * dr;
    }
  }
  if (B > 2 && P->angle_k != 0.0) {
    for (int64_t m = i - 1; m <= i + 1; ++m) { /* middle bead of each angle containing i */
      if (m < 1 || m + 1 >= n) continue;
      if ((m % B) == 0 || (m % B) == B - 1) continue; /* m needs both chain neighbours */
      double fa[3], fm[3], fb[3];
      double v = angle_term(P, &x[3 * (m - 1)], &x[3 * m], &x[3 * (m + 1)], fa, fm, fb);
      const double* fi = (i == m - 1) ? fa : (i == m ? fm : fb);
      for (int k = 0; k < 3; ++k) f[k] += fi[k];
      if (scale) *scale += sqrt(fi[0] * fi[0] + fi[1] * fi[1] + fi[2] * fi[2]);
      ui += v / 3.0;
    }
  }
  if (P->wall_enable && !(con && con[i])) ui += wall_term(P, &x[3 * i], f, scale, bad);
  return ui;
}

/* Bonded and wall forces and energies of all particles (f and u are added
 * to). Returns 1 if a particle is behind a wall. */
int orc_bond_wall_forces(const orc_params* P, int64_t n, const double* x, const int32_t* type,
                         const uint8_t* constrained, double* f, double* u) {
  int bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    double fi[3] = {0.0, 0.0, 0.0};
    double ui = bonded_on(P, n, x, type, constrained, i, fi, NULL, &bad);
    for (int k = 0; k < 3; ++k) f[3 * i + k] += fi[k];
    if (u) u[i] += ui;
  }
  return bad;
}

/* ------------------------------------------------------------------------ */
/* A system advanced by Algorithm S1                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  orc_surface S;
  orc_params P;
  int64_t n;
  uint64_t step;
  double* x;      /* x^k (unwrapped)                    */
  double* p;      /* p^k                                 */
  double* ph;     /* p^{k-1/2}                           */
  double* F;      /* combined force F^k of Algorithm S1  */
  double* fr;     /* random force f_r^k                  */
  double* fc;     /* conservative force at x^k          */
  double* u;      /* per-particle potential energy       */
  double* xref;   /* reference positions for the MSD    */
  int32_t* type;
  int32_t* mol;
  uint8_t* con;
  int64_t newton_fail;     /* particle-steps that missed the tolerance */
  int64_t newton_floor;    /* particle-steps ended at the round-off floor */
  int64_t newton_iters;    /* total Newton iterations of the position half */
  int32_t wall_bad;
} orc_sys;

static double mass_of(const orc_sys* s, int64_t i) { return s->P.mass[s->type[i]]; }

orc_sys* orc_create(const orc_surface* S, const orc_params* P, int64_t n) {
  orc_sys* s = (orc_sys*)calloc(1, sizeof(orc_sys));
  if (!s) return NULL;
  s->S = *S;
  s->P = *P;
  s->n = n;
  size_t n3 = sizeof(double) * 3 * (size_t)(n > 0 ? n : 1);
  s->x = (double*)calloc(1, n3);
  s->p = (double*)calloc(1, n3);
  s->ph = (double*)calloc(1, n3);
  s->F = (double*)calloc(1, n3);
  s->fr = (double*)calloc(1, n3);
  s->fc = (double*)calloc(1, n3);
  s->xref = (double*)calloc(1, n3);
  s->u = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  s->type = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  s->mol = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  s->con = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  return s;
}

void orc_destroy(orc_sys* s) {
  if (!s) return;
  free(s->x); free(s->p); free(s->ph); free(s->F); free(s->fr); free(s->fc);
  free(s->xref); free(s->u); free(s->type); free(s->mol); free(s->con);
  free(s);
}

/* Conservative forces f = -grad V at the current positions into s->fc, s->u. */
int orc_sys_forces(orc_sys* s) {
  int mode = s->P.force_mode;
  if (mode == 0) mode = (s->n <= 4000) ? 1 : 2;
  if (mode == 1)
    orc_pair_forces_brute(&s->P, s->n, s->x, s->type, s->mol, s->fc, s->u);
  else if (orc_pair_forces_cells(&s->P, s->n, s->x, s->type, s->mol, s->fc, s->u))
    return -1;
  if (orc_bond_wall_forces(&s->P, s->n, s->x, s->type, s->con, s->fc, s->u)) s->wall_bad = 1;
  return 0;
}

/* Random force f_r^k of every particle (Algorithm S1):
 * sqrt(2 m kT / (tau dt)) * N(0,1)^3 with 1/tau = gamma. */
static void random_forces(orc_sys* s, uint64_t k, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    double m = mass_of(s, i);
    double amp = sqrt(2.0 * m * s->P.kT * s->P.gamma / s->P.dt);
    double xi[3];
    orc_gauss3(s->P.seed, s->P.replica, (uint32_t)i, k, xi);
    for (int c = 0; c < 3; ++c) out[3 * i + c] = amp * xi[c];
  }
}

/* Set x^k, v^k at step counter k. Returns 1 if a constrained particle is
 * off its surface (|g|/|grad g| >= 1e-6), 2 on an allocation failure. */
int orc_set_state(orc_sys* s, const double* x, const double* v, const int32_t* type,
                  const int32_t* mol, const uint8_t* con, uint64_t step0) {
  int64_t n = s->n;
  for (int64_t i = 0; i < n; ++i) {
    s->type[i] = type ? type[i] : 0;
    if (mol) s->mol[i] = mol[i];
    else s->mol[i] = (int32_t)(s->P.beads_per_mol > 1 ? i / s->P.beads_per_mol : i);
    s->con[i] = con ? con[i] : (uint8_t)(s->S.kind != 0);
    if (s->S.kind == 7) s->con[i] = 0; /* 2D: no constraint, no z motion */
  }
  for (int64_t i = 0; i < n; ++i) {
    double m = mass_of(s, i);
    double vi[3] = {v ? v[3 * i] : 0.0, v ? v[3 * i + 1] : 0.0, v ? v[3 * i + 2] : 0.0};
    for (int k = 0; k < 3; ++k) s->x[3 * i + k] = x[3 * i + k];
    if (s->S.kind == 7) {
      if (!(fabs(x[3 * i + 2] - s->S.c[2]) < 1e-6)) return 1;
      vi[2] = 0.0;
    }
    if (s->con[i]) {
      double nn[3];
      double g = orc_surface_g(&s->S, &s->P, &x[3 * i], nn);
      double n2 = nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2];
      if (!(fabs(g) / sqrt(n2) < 1e-6)) return 1;
      double nv = nn[0] * vi[0] + nn[1] * vi[1] + nn[2] * vi[2];
      for (int k = 0; k < 3; ++k) vi[k] -= nv / n2 * nn[k];
    }
    for (int k = 0; k < 3; ++k) {
      s->p[3 * i + k] = m * vi[k];
      s->ph[3 * i + k] = s->p[3 * i + k];
      s->xref[3 * i + k] = x[3 * i + k];
    }
  }
  s->step = step0;
  if (orc_sys_forces(s)) return 2;
  /* Reading R2: F^{k0} = f(x^{k0}) - gamma p^{k0} + f_r^{k0}. */
  random_forces(s, step0, s->fr);
  for (int64_t i = 0; i < 3 * n; ++i) s->F[i] = s->fc[i] - s->P.gamma * s->p[i] + s->fr[i];
  return 0;
}

/* nsteps of Algorithm S1. Returns the number of particle-steps whose
 * position-half Newton missed the tolerance (0 on success). */
int64_t orc_step(orc_sys* s, int64_t nsteps) {
  int64_t n = s->n;
  int64_t fails = 0;
  double* frn = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  if (!frn) return -1;
  const double dt = s->P.dt, gam = s->P.gamma;
  for (int64_t st = 0; st < nsteps; ++st) {
    /* 1. position update of Algorithm 1 for every particle (the particles
     * are independent: OpenMP threads take disjoint ranges) */
    int64_t n_iters = 0, n_fail = 0, n_floor = 0;
#pragma omp parallel for schedule(static) reduction(+ : n_iters, n_fail, n_floor)
    for (int64_t i = 0; i < n; ++i) {
      double m = mass_of(s, i);
      double* xi = &s->x[3 * i];
      double* pi = &s->p[3 * i];
      double* Fi = &s->F[3 * i];
      if (s->con[i]) {
        double xn[3], phn[3];
        int32_t its = 0;
        int rc = orc_position_half(&s->S, &s->P, xi, pi, Fi, m, xn, phn, NULL, &its);
        n_iters += its;
        if (rc < 0) {
          n_fail++;
        } else if (rc == 1) {
          n_floor++;
        }
        for (int k = 0; k < 3; ++k) {
          xi[k] = xn[k];
          s->ph[3 * i + k] = phn[k];
        }
      } else {
        /* free particle; in the 2D plane the z updates are not evaluated */
        int dims = s->S.kind == 7 ? 2 : 3;
        for (int k = 0; k < dims; ++k) {
          s->ph[3 * i + k] = pi[k] + 0.5 * dt * Fi[k];
          xi[k] += dt / m * s->ph[3 * i + k];
        }
      }
    }
    s->newton_iters += n_iters;
    s->newton_fail += n_fail;
    s->newton_floor += n_floor;
    fails += n_fail;
    s->step += 1;
    /* 2. new conservative forces f^{m+1} = -grad V */
    if (orc_sys_forces(s)) {
      free(frn);
      return -1;
    }
    /* 3. new random force and the combination of Algorithm S1 */
    random_forces(s, s->step, frn);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < 3 * n; ++i) {
      s->F[i] = (s->fc[i] - gam * s->ph[i] + 0.5 * (frn[i] + s->fr[i])) / (1.0 + 0.5 * dt * gam);
      s->fr[i] = frn[i];
    }
    /* 4. momentum update of Algorithm 1 */
    int64_t m_fail = 0;
#pragma omp parallel for schedule(static) reduction(+ : m_fail)
    for (int64_t i = 0; i < n; ++i) {
      double m = mass_of(s, i);
      if (s->con[i]) {
        double pn[3];
        int rc = orc_momentum_half(&s->S, &s->P, &s->x[3 * i], &s->ph[3 * i],
                                   &s->F[3 * i], m, pn, NULL, NULL);
        if (rc < 0) m_fail++;
        for (int k = 0; k < 3; ++k) s->p[3 * i + k] = pn[k];
      } else {
        int dims = s->S.kind == 7 ? 2 : 3;
        for (int k = 0; k < dims; ++k) s->p[3 * i + k] = s->ph[3 * i + k] + 0.5 * dt * s->F[3 * i + k];
      }
    }
    s->newton_fail += m_fail;
    fails += m_fail;
  }
  free(frn);
  return fails;
}

/* Threads of the per-particle loops (1 without OpenMP). The particles'
 * arithmetic, and every sum's order, is the same at any count. */
int orc_set_threads(int k) {
#ifdef _OPENMP
  if (k >= 1) omp_set_num_threads(k);
  return omp_get_max_threads();
#else
  (void)k;
  return 1;
#endif
}

void orc_get_state(const orc_sys* s, double* x, double* v, double* p_half,
                   double* F, uint64_t* step) {
  for (int64_t i = 0; i < s->n; ++i) {
    double m = mass_of(s, i);
    for (int k = 0; k < 3; ++k) {
      if (x) x[3 * i + k] = s->x[3 * i + k];
      if (v) v[3 * i + k] = s->p[3 * i + k] / m;
      if (p_half) p_half[3 * i + k] = s->ph[3 * i + k];
      if (F) F[3 * i + k] = s->F[3 * i + k];
    }
  }
  if (step) *step = s->step;
}

/* Conservative force and per-particle energy at the current x. */
void orc_get_forces(const orc_sys* s, double* f, double* u) {
  for (int64_t i = 0; i < 3 * s->n; ++i)
    if (f) f[i] = s->fc[i];
  for (int64_t i = 0; i < s->n; ++i)
    if (u) u[i] = s->u[i];
}

/* max |g|/|grad g|, max |g|, max |n.v|/|n| over constrained particles. */
void orc_residual(const orc_sys* s, double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  for (int64_t i = 0; i < s->n; ++i) {
    if (!s->con[i]) continue;
    double nn[3];
    double g = orc_surface_g(&s->S, &s->P, &s->x[3 * i], nn);
    double gn = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    double m = mass_of(s, i);
    double nv = (nn[0] * s->p[3 * i] + nn[1] * s->p[3 * i + 1] + nn[2] * s->p[3 * i + 2]) / m;
    if (fabs(g) / gn > out[0]) out[0] = fabs(g) / gn;
    if (fabs(g) > out[1]) out[1] = fabs(g);
    if (fabs(nv) / gn > out[2]) out[2] = fabs(nv) / gn;
  }
}

/* Observables (Section 3.1, SI S1.3): out = {K, U, kT, msd, r0.rt/R^2, ndof}. */
void orc_observables(const orc_sys* s, double out[6]) {
  double K = 0.0, U = 0.0, msd = 0.0, rr = 0.0;
  int64_t ndof = 0;
  for (int64_t i = 0; i < s->n; ++i) {
    double m = mass_of(s, i);
    double p2 = 0.0, d2 = 0.0, dot = 0.0;
    for (int k = 0; k < 3; ++k) {
      p2 += s->p[3 * i + k] * s->p[3 * i + k];
      double d = s->x[3 * i + k] - s->xref[3 * i + k];
      d2 += d * d;
      dot += (s->xref[3 * i + k] - s->S.c[k]) * (s->x[3 * i + k] - s->S.c[k]);
    }
    K += p2 / (2.0 * m);
    U += s->u[i];
    msd += d2;
    rr += dot;
    ndof += (s->con[i] || s->S.kind == 7) ? 2 : 3;
  }
  out[0] = K;
  out[1] = U;
  out[2] = ndof > 0 ? 2.0 * K / (double)ndof : 0.0;
  out[3] = s->n > 0 ? msd / (double)s->n : 0.0;
  out[4] = (s->S.kind == 2 && s->n > 0) ? rr / (double)s->n / (s->S.p[0] * s->S.p[0]) : 0.0;
  out[5] = (double)ndof;
}

/* Newton statistics: {failures, round-off-floor exits, total iterations}. */
void orc_newton_stats(const orc_sys* s, int64_t out[3]) {
  out[0] = s->newton_fail;
  out[1] = s->newton_floor;
  out[2] = s->newton_iters;
}

int32_t orc_wall_violation(const orc_sys* s) { return s->wall_bad; }

/* ------------------------------------------------------------------------ */
/* One particle at a time (sampled checks of large systems)                  */
/* ------------------------------------------------------------------------ */
/* Conservative force and energy on particle i of a system of n particles:
 * every pair (i, j) of Eq. (S1) with the minimum image, plus its bonds and
 * walls (readings R5, R6). O(n). */
void orc_force_on(const orc_params* P, int64_t n, const double* x, const int32_t* type,
                  const int32_t* mol, const uint8_t* con, int64_t i, double f[3], double* u) {
  f[0] = f[1] = f[2] = 0.0;
  double ui = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    if (j == i || same_molecule(P, mol, i, j)) continue;
    double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
    min_image(P, d);
    ui += 0.5 * lj_pair(P, type[i], type[j], d, f);
  }
  ui += bonded_on(P, n, x, type, con, i, f, NULL, NULL);
  if (u) *u = ui;
}

/* Algorithm S1 for one particle i whose neighbours sit at x (all n):
 * from p_in (p^k when first = 1, else p^{k-1/2}) at step counter k, form the
 * force f^k, the random force and the combined force F^k (reading R2 when
 * first = 1), the momentum half (when first = 0) giving p^k, then the
 * position half of the next step giving x^{k+1} and p^{k+1/2}. Returns the
 * position-half status of orc_position_half (0 for a free particle). */
int orc_particle_advance(const orc_surface* S, const orc_params* P, int64_t n, const double* x,
                         const int32_t* type, const int32_t* mol, const uint8_t* con, int64_t i,
                         const double p_in[3], uint64_t k, int first, double p_k[3],
                         double x_new[3], double p_half_new[3]) {
  double m = P->mass[type[i]];
  double f[3];
  orc_force_on(P, n, x, type, mol, con, i, f, NULL);
  double amp = sqrt(2.0 * m * P->kT * P->gamma / P->dt);
  double xk[3], xkm1[3];
  orc_gauss3(P->seed, P->replica, (uint32_t)i, k, xk);
  double F[3];
  if (first) {
    for (int c = 0; c < 3; ++c) {
      F[c] = f[c] - P->gamma * p_in[c] + amp * xk[c];
      p_k[c] = p_in[c];
    }
  } else {
    orc_gauss3(P->seed, P->replica, (uint32_t)i, k - 1, xkm1);
    for (int c = 0; c < 3; ++c)
      F[c] = (f[c] - P->gamma * p_in[c] + 0.5 * amp * (xk[c] + xkm1[c])) / (1.0 + 0.5 * P->dt * P->gamma);
    if (con && con[i]) {
      if (orc_momentum_half(S, P, &x[3 * i], p_in, F, m, p_k, NULL, NULL) < 0) return -1;
    } else {
      for (int c = 0; c < 3; ++c) p_k[c] = p_in[c] + 0.5 * P->dt * F[c];
    }
  }
  if (con && con[i])
    return orc_position_half(S, P, &x[3 * i], p_k, F, m, x_new, p_half_new, NULL, NULL);
  for (int c = 0; c < 3; ++c) {
    p_half_new[c] = p_k[c] + 0.5 * P->dt * F[c];
    x_new[c] = x[3 * i + c] + P->dt / m * p_half_new[c];
  }
  return 0;
}

/* Force scale of every particle: sum over its pair, bond and wall terms of
 * the magnitude of each term's force (the size of the numbers whose sum is
 * the particle's force). Brute force over all pairs. */
void orc_force_scale(const orc_params* P, int64_t n, const double* x, const int32_t* type,
                     const int32_t* mol, const uint8_t* con, double* scale) {
  memset(scale, 0, sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      if (j == i || same_molecule(P, mol, i, j)) continue;
      double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
      min_image(P, d);
      double fi[3] = {0.0, 0.0, 0.0};
      lj_pair(P, type[i], type[j], d, fi);
      scale[i] += sqrt(fi[0] * fi[0] + fi[1] * fi[1] + fi[2] * fi[2]);
    }
  }
  /* bonds, angles and walls: add |f| of each term */
  for (int64_t i = 0; i < n; ++i) {
    double fi[3] = {0.0, 0.0, 0.0};
    bonded_on(P, n, x, type, con, i, fi, &scale[i], NULL);
  }
}
