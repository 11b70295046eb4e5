/*
 * nbody_oracle.c -- the reference ("oracle") for the direct-sum N-body method
 * with velocity-Verlet integration studied in arXiv:2112.15079.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * CPU statement of what the CUDA library computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, constant or helper with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Arithmetic: IEEE binary64 throughout.  Build with -O2 -ffp-contract=off
 * and without -ffast-math, so every expression rounds exactly as written.
 * An optional -fopenmp build parallelises only the outer loop over target
 * bodies p; each p owns its accumulator and visits j in ascending order, so
 * that build is bitwise identical to the single-threaded one.
 *
 * Notation (paper Section 2): bodies p, j = 0..n-1, position r_p = (x,y,z),
 * mass m_j, gravitational constant G, step size dt.  "Eq. 1" is the
 * direct-sum acceleration, "Eq. 3"/"Eq. 4" the velocity-Verlet position and
 * velocity updates.  The paper uses no softening; the pair j == p is left out
 * by its index, as the sum in Eq. 1 states.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Neumaier's compensated summation: running (sum, compensation). */
static void neumaier_add(double *sum, double *comp, double v) {
  const double t = *sum + v;
  if (fabs(*sum) >= fabs(v))
    *comp += (*sum - t) + v;
  else
    *comp += (v - t) + *sum;
  *sum = t;
}

/* Eq. 1: acceleration of body p,
 *   a_p = sum_{j != p} G m_j (r_j - r_p) / |r_j - r_p|^3,
 * summed over j in ascending order with Neumaier compensation, so the
 * result is the exact sum of the rounded terms to about one ulp.  (A plain
 * running sum is not: for a moon, ~1e4 asteroid terms 1e-8 times smaller
 * than its host's pull round the same way and drift by ~3e-13 relative.)
 * rows: the target bodies to evaluate (n_rows of them, out arrays indexed
 * like rows); rows == NULL means all n. */
static void accel_rows(int64_t n, double G, const double *x, const double *y,
                       const double *z, const double *m, int64_t n_rows,
                       const int64_t *rows, double *ax, double *ay,
                       double *az) {
  int64_t k;
#pragma omp parallel for schedule(dynamic, 16)
  for (k = 0; k < n_rows; k++) {
    const int64_t p = rows ? rows[k] : k;
    double sx = 0.0, sy = 0.0, sz = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
    for (int64_t j = 0; j < n; j++) {
      if (j == p) continue;
      const double dx = x[j] - x[p];
      const double dy = y[j] - y[p];
      const double dz = z[j] - z[p];
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double s = 1.0 / (r2 * sqrt(r2)); /* |d|^-3 */
      const double f = G * m[j] * s;
      neumaier_add(&sx, &cx, f * dx);
      neumaier_add(&sy, &cy, f * dy);
      neumaier_add(&sz, &cz, f * dz);
    }
    ax[k] = sx + cx;
    ay[k] = sy + cy;
    az[k] = sz + cz;
  }
}

/* Eq. 1 for every body. */
void oracle_accel(int64_t n, double G, const double *x, const double *y,
                  const double *z, const double *m, double *ax, double *ay,
                  double *az) {
  accel_rows(n, G, x, y, z, m, n, NULL, ax, ay, az);
}

/* Eq. 1 for the listed target bodies only (sampled rows at large n). */
void oracle_accel_rows(int64_t n, double G, const double *x, const double *y,
                       const double *z, const double *m, int64_t n_rows,
                       const int64_t *rows, double *ax, double *ay,
                       double *az) {
  accel_rows(n, G, x, y, z, m, n_rows, rows, ax, ay, az);
}

/* Sum of the magnitudes of the terms of Eq. 1 for the listed targets,
 *   T_p = sum_{j != p} G m_j / |r_j - r_p|^2,
 * the scale against which a rounding error in a_p is judged when the terms
 * cancel (condition number of the sum = T_p / |a_p|). */
void oracle_term_norm_rows(int64_t n, double G, const double *x,
                           const double *y, const double *z, const double *m,
                           int64_t n_rows, const int64_t *rows, double *t) {
  int64_t k;
#pragma omp parallel for schedule(dynamic, 16)
  for (k = 0; k < n_rows; k++) {
    const int64_t p = rows ? rows[k] : k;
    double s = 0.0;
    for (int64_t j = 0; j < n; j++) {
      if (j == p) continue;
      const double dx = x[j] - x[p];
      const double dy = y[j] - y[p];
      const double dz = z[j] - z[p];
      s += G * m[j] / (dx * dx + dy * dy + dz * dz);
    }
    t[k] = s;
  }
}

/* Eqs. 3-4, n_steps velocity-Verlet steps of size dt, in place.
 * On entry (ax,ay,az) must hold a_i = Eq. 1 evaluated at the entry
 * positions; on return it holds the acceleration at the returned positions.
 * Per step:
 *   Eq. 3: r_{i+1} = r_i + v_i dt + (1/2) a_i dt^2
 *   Eq. 1: a_{i+1} = A(r_{i+1})
 *   Eq. 4: v_{i+1} = v_i + (1/2) (a_i + a_{i+1}) dt
 * Returns 0, or -1 if scratch could not be allocated. */
int oracle_verlet(int64_t n, double G, double dt, int64_t n_steps, double *x,
                  double *y, double *z, double *vx, double *vy, double *vz,
                  const double *m, double *ax, double *ay, double *az) {
  double *nx = (double *)malloc(sizeof(double) * (size_t)(3 * n > 0 ? 3 * n : 1));
  if (!nx) return -1;
  double *ny = nx + n, *nz = nx + 2 * n;
  const double h = 0.5 * dt * dt;
  for (int64_t step = 0; step < n_steps; step++) {
    for (int64_t p = 0; p < n; p++) { /* Eq. 3 */
      x[p] = x[p] + vx[p] * dt + h * ax[p];
      y[p] = y[p] + vy[p] * dt + h * ay[p];
      z[p] = z[p] + vz[p] * dt + h * az[p];
    }
    oracle_accel(n, G, x, y, z, m, nx, ny, nz); /* Eq. 1 */
    for (int64_t p = 0; p < n; p++) { /* Eq. 4 */
      vx[p] = vx[p] + 0.5 * (ax[p] + nx[p]) * dt;
      vy[p] = vy[p] + 0.5 * (ay[p] + ny[p]) * dt;
      vz[p] = vz[p] + 0.5 * (az[p] + nz[p]) * dt;
      ax[p] = nx[p];
      ay[p] = ny[p];
      az[p] = nz[p];
    }
  }
  free(nx);
  return 0;
}

/* The leapfrog method Section 2 names beside Verlet, in its
 * drift-kick-drift form: the force is taken at the half-step positions,
 *   r_{n+1/2} = r_n + (dt/2) v_n,
 *   v_{n+1}   = v_n + dt A(r_{n+1/2}),
 *   r_{n+1}   = r_{n+1/2} + (dt/2) v_{n+1},
 * so positions and velocities are reported at the same (integer) times.
 * One evaluation of Eq. 1 per step; on return (ax, ay, az) = A at the last
 * half-step positions.  Returns 0, or -1 if scratch could not be allocated. */
int oracle_leapfrog(int64_t n, double G, double dt, int64_t n_steps, double *x,
                    double *y, double *z, double *vx, double *vy, double *vz,
                    const double *m, double *ax, double *ay, double *az) {
  double *r[3] = {x, y, z}, *v[3] = {vx, vy, vz}, *a[3] = {ax, ay, az};
  const double h = 0.5 * dt;
  for (int64_t step = 0; step < n_steps; step++) {
    for (int k = 0; k < 3; k++) /* drift half a step */
      for (int64_t p = 0; p < n; p++) r[k][p] = r[k][p] + h * v[k][p];
    oracle_accel(n, G, x, y, z, m, ax, ay, az); /* Eq. 1 at r_{n+1/2} */
    for (int k = 0; k < 3; k++)
      for (int64_t p = 0; p < n; p++) {
        v[k][p] = v[k][p] + dt * a[k][p]; /* kick a full step */
        r[k][p] = r[k][p] + h * v[k][p]; /* drift the other half */
      }
  }
  return 0;
}

/* The fourth-order Runge-Kutta method that Section 2 names as the
 * higher-order alternative to Verlet, applied to the first-order system
 * y = (r, v), y' = f(y) = (v, A(r)) with A = Eq. 1, n_steps steps of dt:
 *   k1 = f(y),  k2 = f(y + dt/2 k1),  k3 = f(y + dt/2 k2),  k4 = f(y + dt k3),
 *   y <- y + dt/6 (k1 + 2 k2 + 2 k3 + k4).
 * Four evaluations of Eq. 1 per step.  On return (ax, ay, az) = A(r) at the
 * final positions.  Returns 0, or -1 if scratch could not be allocated. */
int oracle_rk4(int64_t n, double G, double dt, int64_t n_steps, double *x,
               double *y, double *z, double *vx, double *vy, double *vz,
               const double *m, double *ax, double *ay, double *az) {
  /* scratch: stage position (3n), stage velocity (3n), stage acceleration
   * (3n), and the weighted sums of the stage derivatives for r and v (6n) */
  const size_t n3 = (size_t)(3 * n > 0 ? 3 * n : 1);
  double *buf = (double *)malloc(sizeof(double) * 5 * n3);
  if (!buf) return -1;
  double *sr = buf, *sv = buf + n3, *sa = buf + 2 * n3, *dr = buf + 3 * n3,
         *dv = buf + 4 * n3;
  double *r[3] = {x, y, z}, *v[3] = {vx, vy, vz};
  const double c_stage[4] = {0.0, 0.5, 0.5, 1.0}; /* where k_s is taken */
  const double w_stage[4] = {1.0, 2.0, 2.0, 1.0}; /* its weight (/6) */
  for (int64_t step = 0; step < n_steps; step++) {
    for (size_t i = 0; i < 3 * (size_t)n; i++) dr[i] = dv[i] = 0.0;
    for (int s = 0; s < 4; s++) {
      /* stage state y + c_s dt k_{s-1}, with k_{s-1} = (sv, sa) */
      for (int k = 0; k < 3; k++)
        for (int64_t p = 0; p < n; p++) {
          const size_t i = (size_t)k * n + p;
          if (s == 0) {
            sr[i] = r[k][p];
            sv[i] = v[k][p];
          } else {
            const double kr = sv[i], kv = sa[i];
            sr[i] = r[k][p] + c_stage[s] * dt * kr;
            sv[i] = v[k][p] + c_stage[s] * dt * kv;
          }
        }
      oracle_accel(n, G, sr, sr + n, sr + 2 * n, m, sa, sa + n, sa + 2 * n);
      /* k_s = (sv, sa) */
      for (size_t i = 0; i < 3 * (size_t)n; i++) {
        dr[i] += w_stage[s] * sv[i];
        dv[i] += w_stage[s] * sa[i];
      }
    }
    for (int k = 0; k < 3; k++)
      for (int64_t p = 0; p < n; p++) {
        const size_t i = (size_t)k * n + p;
        r[k][p] = r[k][p] + dt / 6.0 * dr[i];
        v[k][p] = v[k][p] + dt / 6.0 * dv[i];
      }
  }
  oracle_accel(n, G, x, y, z, m, ax, ay, az);
  free(buf);
  return 0;
}

/* Total energy, the accuracy criterion of Section 2 and Section 4:
 *   E_kin = sum_p (1/2) m_p |v_p|^2
 *   E_pot = - sum_{p < j} G m_p m_j / |r_j - r_p|
 * Both sums use Neumaier summation, pairs visited p ascending then j > p
 * ascending. */
void oracle_energy(int64_t n, double G, const double *x, const double *y,
                   const double *z, const double *vx, const double *vy,
                   const double *vz, const double *m, double *e_kin,
                   double *e_pot) {
  double ks = 0.0, kc = 0.0, ps = 0.0, pc = 0.0;
  for (int64_t p = 0; p < n; p++) {
    const double v2 = vx[p] * vx[p] + vy[p] * vy[p] + vz[p] * vz[p];
    neumaier_add(&ks, &kc, 0.5 * m[p] * v2);
  }
  for (int64_t p = 0; p < n; p++) {
    for (int64_t j = p + 1; j < n; j++) {
      const double dx = x[j] - x[p];
      const double dy = y[j] - y[p];
      const double dz = z[j] - z[p];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      neumaier_add(&ps, &pc, -(G * m[p] * m[j] / r));
    }
  }
  *e_kin = ks + kc;
  *e_pot = ps + pc;
}

/* Vector-Jacobian product of Eq. 1, accumulated into (rx,ry,rz) and gm.
 * With d = r_j - r_q and the pair kernel f(d) = d / |d|^3, the Jacobian of f
 * is the symmetric 3x3 matrix
 *   K(d) = I / |d|^3 - 3 d d^T / |d|^5,        K(-d) = K(d).
 * dA_p/dr_q = G m_q K(r_q - r_p) for q != p and -G sum_j m_j K(r_j - r_p)
 * for q == p, so for an adjoint vector w on the accelerations
 *   (J^T w)_q  = G sum_{j != q} K(r_j - r_q) (m_q w_j - m_j w_q),
 *   (dA/dm)^T w at q = G sum_{p != q} w_p . (r_q - r_p) / |r_q - r_p|^3.
 * K is formed explicitly per pair, j ascending.
 * With W = (Wx, Wy, Wz) non-NULL (elementwise magnitudes bounding |w|), the
 * same loop also accumulates the magnitudes of every term of both sums into
 * (Rx, Ry, Rz) and Gm:
 *   G sum_{j != q} |K(d)| (m_q W_j + m_j W_q)   (|K| elementwise),
 *   G sum_{p != q} W_p . |r_q - r_p| / |r_q - r_p|^3   (|.| elementwise). */
static void vjp_impl(int64_t n, double G, const double *x, const double *y,
                     const double *z, const double *m, const double *wx,
                     const double *wy, const double *wz, double *rx,
                     double *ry, double *rz, double *gm, const double *Wx,
                     const double *Wy, const double *Wz, double *Rx,
                     double *Ry, double *Rz, double *Gm) {
  int64_t q;
#pragma omp parallel for schedule(dynamic, 16)
  for (q = 0; q < n; q++) {
    double sx = 0.0, sy = 0.0, sz = 0.0, sm = 0.0;
    double ax = 0.0, ay = 0.0, az = 0.0, am = 0.0;
    for (int64_t j = 0; j < n; j++) {
      if (j == q) continue;
      const double d[3] = {x[j] - x[q], y[j] - y[q], z[j] - z[q]};
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      const double r = sqrt(r2);
      const double i3 = 1.0 / (r2 * r); /* |d|^-3 */
      const double i5 = i3 / r2;        /* |d|^-5 */
      double K[3][3];
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
          K[a][b] = (a == b ? i3 : 0.0) - 3.0 * d[a] * d[b] * i5;
      const double u[3] = {m[q] * wx[j] - m[j] * wx[q],
                           m[q] * wy[j] - m[j] * wy[q],
                           m[q] * wz[j] - m[j] * wz[q]};
      sx += G * (K[0][0] * u[0] + K[0][1] * u[1] + K[0][2] * u[2]);
      sy += G * (K[1][0] * u[0] + K[1][1] * u[1] + K[1][2] * u[2]);
      sz += G * (K[2][0] * u[0] + K[2][1] * u[1] + K[2][2] * u[2]);
      /* w_j . (r_q - r_j) |r_q - r_j|^-3 = -(w_j . d) i3 */
      sm += -G * (wx[j] * d[0] + wy[j] * d[1] + wz[j] * d[2]) * i3;
      if (Wx) {
        const double U[3] = {m[q] * Wx[j] + m[j] * Wx[q],
                             m[q] * Wy[j] + m[j] * Wy[q],
                             m[q] * Wz[j] + m[j] * Wz[q]};
        ax += G * (fabs(K[0][0]) * U[0] + fabs(K[0][1]) * U[1] + fabs(K[0][2]) * U[2]);
        ay += G * (fabs(K[1][0]) * U[0] + fabs(K[1][1]) * U[1] + fabs(K[1][2]) * U[2]);
        az += G * (fabs(K[2][0]) * U[0] + fabs(K[2][1]) * U[1] + fabs(K[2][2]) * U[2]);
        am += G * (Wx[j] * fabs(d[0]) + Wy[j] * fabs(d[1]) + Wz[j] * fabs(d[2])) * i3;
      }
    }
    rx[q] += sx;
    ry[q] += sy;
    rz[q] += sz;
    gm[q] += sm;
    if (Wx) {
      Rx[q] += ax;
      Ry[q] += ay;
      Rz[q] += az;
      Gm[q] += am;
    }
  }
}

void oracle_vjp(int64_t n, double G, const double *x, const double *y,
                const double *z, const double *m, const double *wx,
                const double *wy, const double *wz, double *rx, double *ry,
                double *rz, double *gm) {
  vjp_impl(n, G, x, y, z, m, wx, wy, wz, rx, ry, rz, gm, NULL, NULL, NULL,
           NULL, NULL, NULL, NULL);
}

/* Gradient of a loss L(r_T, v_T) with respect to (r_0, v_0, m) through T
 * velocity-Verlet steps (Eqs. 1, 3, 4), by the discrete adjoint of exactly
 * that recurrence.  Reverse sweep, adjoints rho = dL/dr, nu = dL/dv,
 * alpha = dL/da:
 *   start rho = dL/dr_T, nu = dL/dv_T, alpha = 0;
 *   for i = T-1 .. 0:
 *     alpha += dt/2 nu                 (Eq. 4 of step i feeds a_{i+1})
 *     rho += J(r_{i+1})^T alpha;  gm += (dA/dm)(r_{i+1})^T alpha
 *     (rho, nu, alpha) <- (rho, nu + dt rho, dt/2 nu + dt^2/2 rho)
 *                                      (Eq. 3 and Eq. 4 of step i)
 *   finally rho += J(r_0)^T alpha;  gm += (dA/dm)(r_0)^T alpha.
 * The forward trajectory r_0..r_T is stored whole (no checkpointing).
 * dLdv_T may be NULL (zero).  Outputs are 3n (x block, y block, z block),
 * 3n and n doubles.
 * absr, absv, absm (all NULL, or 3n, 3n, n outputs): the scale against
 * which a rounding error in each gradient element is judged -- the sum of
 * the magnitudes of everything the sweep adds into that element: for rho,
 * |dL/dr_T| plus, at every product, the magnitudes of the terms of J^T alpha
 * (vjp_impl's magnitude form with the sweep's own alpha); for g_m the
 * magnitudes of the mass terms likewise; for nu, |dL/dv_T| plus, at every
 * update nu += dt rho, |dt| times the bound on |rho| so far.  Each bounds
 * the magnitude of its element (|grad| <= abs elementwise), and abs / |grad|
 * is the element's condition number with respect to errors in the terms.
 * Returns 0, or -1 if memory could not be allocated. */
int oracle_grad(int64_t n, double G, double dt, int64_t T, const double *x0,
                const double *y0, const double *z0, const double *vx0,
                const double *vy0, const double *vz0, const double *m,
                const double *dLdr_T, const double *dLdv_T, double *dLdr0,
                double *dLdv0, double *dLdm, double *absr, double *absv,
                double *absm) {
  const size_t N = (size_t)n;
  const int mag = absr != NULL && absv != NULL && absm != NULL;
  double *traj = (double *)malloc(sizeof(double) * 3 * N * (size_t)(T + 1));
  double *work = (double *)malloc(sizeof(double) * 9 * N + 8);
  double *mw = mag ? (double *)malloc(sizeof(double) * 3 * N + 8) : NULL;
  if (!traj || !work || (mag && !mw)) {
    free(traj);
    free(work);
    free(mw);
    return -1;
  }
  double *x = work, *y = work + N, *z = work + 2 * N;
  double *vx = work + 3 * N, *vy = work + 4 * N, *vz = work + 5 * N;
  double *ax = work + 6 * N, *ay = work + 7 * N, *az = work + 8 * N;
  memcpy(x, x0, sizeof(double) * N);
  memcpy(y, y0, sizeof(double) * N);
  memcpy(z, z0, sizeof(double) * N);
  memcpy(vx, vx0, sizeof(double) * N);
  memcpy(vy, vy0, sizeof(double) * N);
  memcpy(vz, vz0, sizeof(double) * N);
  oracle_accel(n, G, x, y, z, m, ax, ay, az);
  for (int64_t i = 0; i <= T; i++) {
    double *r = traj + 3 * N * (size_t)i;
    memcpy(r, x, sizeof(double) * N);
    memcpy(r + N, y, sizeof(double) * N);
    memcpy(r + 2 * N, z, sizeof(double) * N);
    if (i < T &&
        oracle_verlet(n, G, dt, 1, x, y, z, vx, vy, vz, m, ax, ay, az) != 0) {
      free(traj);
      free(work);
      return -1;
    }
  }
  /* reuse work as (nu, alpha, nu_next); magnitudes: absr, absv, absm
   * accumulate; A = |alpha| (scratch in mw) */
  double *nu = work, *al = work + 3 * N, *tmp = work + 6 * N;
  double *rho = dLdr0;
  double *A = mw;
  const double adt = fabs(dt);
  memcpy(rho, dLdr_T, sizeof(double) * 3 * N);
  if (dLdv_T)
    memcpy(nu, dLdv_T, sizeof(double) * 3 * N);
  else
    memset(nu, 0, sizeof(double) * 3 * N);
  memset(al, 0, sizeof(double) * 3 * N);
  memset(dLdm, 0, sizeof(double) * N);
  if (mag) {
    for (size_t k = 0; k < 3 * N; k++) {
      absr[k] = fabs(dLdr_T[k]);
      absv[k] = dLdv_T ? fabs(dLdv_T[k]) : 0.0;
    }
    memset(absm, 0, sizeof(double) * N);
  }
  for (int64_t i = T - 1; i >= 0; i--) {
    for (size_t k = 0; k < 3 * N; k++) al[k] += 0.5 * dt * nu[k];
    if (mag)
      for (size_t k = 0; k < 3 * N; k++) A[k] = fabs(al[k]);
    const double *r = traj + 3 * N * (size_t)(i + 1);
    vjp_impl(n, G, r, r + N, r + 2 * N, m, al, al + N, al + 2 * N, rho,
             rho + N, rho + 2 * N, dLdm, A, A ? A + N : NULL,
             A ? A + 2 * N : NULL, absr, absr ? absr + N : NULL,
             absr ? absr + 2 * N : NULL, absm);
    for (size_t k = 0; k < 3 * N; k++) {
      tmp[k] = nu[k] + dt * rho[k];
      al[k] = 0.5 * dt * nu[k] + 0.5 * dt * dt * rho[k];
    }
    memcpy(nu, tmp, sizeof(double) * 3 * N);
    if (mag)
      for (size_t k = 0; k < 3 * N; k++) absv[k] += adt * absr[k];
  }
  if (mag)
    for (size_t k = 0; k < 3 * N; k++) A[k] = fabs(al[k]);
  vjp_impl(n, G, traj, traj + N, traj + 2 * N, m, al, al + N, al + 2 * N,
           rho, rho + N, rho + 2 * N, dLdm, A, A ? A + N : NULL,
           A ? A + 2 * N : NULL, absr, absr ? absr + N : NULL,
           absr ? absr + 2 * N : NULL, absm);
  memcpy(dLdv0, nu, sizeof(double) * 3 * N);
  free(traj);
  free(work);
  free(mw);
  return 0;
}

/* ------------------------------------------------------------------------
 * Close-encounter handling: impulse multiple time stepping of close pairs.
 *
 * An extension beyond Section 2's method, for bodies whose two-body orbit
 * the fixed step cannot follow (a moon with a period below a few dt is
 * unstable under Eqs. 3-4 at any precision).  It is the reversible impulse
 * multiple-time-step scheme of Tuckerman, Berne and Martyna (J. Chem. Phys.
 * 97, 1990, 1992) with the force split by pairs:
 *
 *   close pair (p, j), p < j:  G (m_p + m_j) dt^2 > theta_c^2 d^3,
 *     d = |r_j - r_p| at the positions the run starts from, i.e. the pair's
 *     two-body angular frequency w = sqrt(G (m_p + m_j) / d^3) has
 *     w dt > theta_c;
 *   cluster: a connected set of bodies joined by close pairs;
 *   sub-steps of a cluster: k = max over its pairs of ceil(w dt / theta_s);
 *   A_near(r)_p = sum over the close pairs (p, j), j ascending, of
 *     G m_j (r_j - r_p) / |r_j - r_p|^3;
 *   A_far(r)_p = the same sum over every other j != p (Eq. 1 without p's
 *     close partners), summed directly rather than as A - A_near, so a
 *     moon's far force does not inherit the rounding of its host's pull.
 *
 * One step of dt:
 *   v <- v + dt/2 A_far(r)                                   every body
 *   r <- r + dt v                                            bodies in no cluster
 *   k times, h = dt / k:  v <- v + h/2 A_near(r); r <- r + h v;
 *                         v <- v + h/2 A_near(r)             each cluster
 *   v <- v + dt/2 A_far(r)                                   every body
 * (A_far = A for a body with no close pair.)
 * Without close pairs this is velocity Verlet in its kick-drift-kick form,
 * algebraically Eqs. 3-4.  The pairs and sub-step counts are fixed when the
 * run starts.  On return (ax, ay, az) = A(r) (Eq. 1) at the final positions;
 * *n_pairs and *k_max (either may be NULL) report the close pairs and the
 * largest sub-step count.  Returns 0; -1 if scratch could not be allocated;
 * -2 if a cluster would need more than 1e6 sub-steps per step.
 * ---------------------------------------------------------------------- */
static int64_t uf_find(int64_t *parent, int64_t i) {
  while (parent[i] != i) {
    parent[i] = parent[parent[i]];
    i = parent[i];
  }
  return i;
}

/* A_near for the bodies listed in idx[0..cnt) (their close partners given as
 * the CSR lists nb_off / nb_j, j ascending). */
static void near_accel(double G, const double *x, const double *y,
                       const double *z, const double *m, const int64_t *idx,
                       int64_t cnt, const int64_t *nb_off, const int64_t *nb_j,
                       double *anx, double *any, double *anz) {
  for (int64_t k = 0; k < cnt; k++) {
    const int64_t p = idx[k];
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t e = nb_off[p]; e < nb_off[p + 1]; e++) {
      const int64_t j = nb_j[e];
      const double dx = x[j] - x[p];
      const double dy = y[j] - y[p];
      const double dz = z[j] - z[p];
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double f = G * m[j] * (1.0 / (r2 * sqrt(r2))); /* as in Eq. 1 above */
      sx += f * dx;
      sy += f * dy;
      sz += f * dz;
    }
    anx[p] = sx;
    any[p] = sy;
    anz[p] = sz;
  }
}

/* A_far for the bodies idx[0..cnt): Eq. 1 over every j != p that is not one
 * of p's close partners (nb_j[nb_off[p] .. nb_off[p+1]), ascending), j
 * ascending, Neumaier-compensated as accel_rows. */
static void far_accel(int64_t n, double G, const double *x, const double *y,
                      const double *z, const double *m, const int64_t *idx,
                      int64_t cnt, const int64_t *nb_off, const int64_t *nb_j,
                      double *fx, double *fy, double *fz) {
  for (int64_t k = 0; k < cnt; k++) {
    const int64_t p = idx[k];
    double sx = 0.0, sy = 0.0, sz = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
    int64_t e = nb_off[p];
    for (int64_t j = 0; j < n; j++) {
      if (j == p) continue;
      while (e < nb_off[p + 1] && nb_j[e] < j) e++;
      if (e < nb_off[p + 1] && nb_j[e] == j) continue; /* a close partner */
      const double dx = x[j] - x[p];
      const double dy = y[j] - y[p];
      const double dz = z[j] - z[p];
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double s = 1.0 / (r2 * sqrt(r2));
      const double f = G * m[j] * s;
      neumaier_add(&sx, &cx, f * dx);
      neumaier_add(&sy, &cy, f * dy);
      neumaier_add(&sz, &cz, f * dz);
    }
    fx[p] = sx + cx;
    fy[p] = sy + cy;
    fz[p] = sz + cz;
  }
}

int oracle_respa(int64_t n, double G, double dt, int64_t n_steps,
                 double theta_c, double theta_s, double *x, double *y,
                 double *z, double *vx, double *vy, double *vz,
                 const double *m, double *ax, double *ay, double *az,
                 int64_t *n_pairs, int64_t *k_max) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * nn);
  int64_t *deg = (int64_t *)calloc(nn + 1, sizeof(int64_t));
  double *wmax = (double *)calloc(nn, sizeof(double));
  double *scratch = (double *)malloc(sizeof(double) * 6 * nn);
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * nn);
  int64_t *kc = (int64_t *)malloc(sizeof(int64_t) * nn);
  if (!parent || !deg || !wmax || !scratch || !order || !kc) {
    free(parent); free(deg); free(wmax); free(scratch); free(order); free(kc);
    return -1;
  }
  double *anx = scratch, *any = scratch + n, *anz = scratch + 2 * n;
  double *fx = scratch + 3 * n, *fy = scratch + 4 * n, *fz = scratch + 5 * n;
  /* close pairs, by brute force over all p < j */
  int64_t pairs = 0;
  for (int64_t p = 0; p < n; p++) parent[p] = p;
  for (int64_t p = 0; p < n; p++)
    for (int64_t j = p + 1; j < n; j++) {
      const double dx = x[j] - x[p], dy = y[j] - y[p], dz = z[j] - z[p];
      const double d2 = dx * dx + dy * dy + dz * dz;
      const double d3 = d2 * sqrt(d2);
      if (G * (m[p] + m[j]) * (dt * dt) > theta_c * theta_c * d3) {
        pairs++;
        deg[p + 1]++;
        deg[j + 1]++;
        parent[uf_find(parent, p)] = uf_find(parent, j);
      }
    }
  for (int64_t p = 0; p < n; p++) deg[p + 1] += deg[p];
  int64_t *nb_j = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * pairs > 0 ? 2 * pairs : 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * nn);
  if (!nb_j || !fill) {
    free(parent); free(deg); free(wmax); free(scratch); free(order); free(kc);
    free(nb_j); free(fill);
    return -1;
  }
  for (int64_t p = 0; p < n; p++) fill[p] = deg[p];
  for (int64_t p = 0; p < n; p++) /* partners in ascending order */
    for (int64_t j = 0; j < n; j++) {
      if (j == p) continue;
      /* the same test as above, on the pair taken as (lower, higher) index */
      const int64_t lo = p < j ? p : j, hi = p < j ? j : p;
      const double dx = x[hi] - x[lo], dy = y[hi] - y[lo], dz = z[hi] - z[lo];
      const double d2 = dx * dx + dy * dy + dz * dz;
      const double d3 = d2 * sqrt(d2);
      if (G * (m[lo] + m[hi]) * (dt * dt) > theta_c * theta_c * d3) {
        nb_j[fill[p]++] = j;
        const double w = sqrt(G * (m[lo] + m[hi]) / d3);
        if (w > wmax[p]) wmax[p] = w;
      }
    }
  /* sub-steps per cluster: the largest w dt / theta_s over its pairs */
  int64_t kmx = 0;
  for (int64_t p = 0; p < n; p++) kc[p] = 0;
  for (int64_t p = 0; p < n; p++) {
    if (deg[p + 1] == deg[p]) continue;
    const int64_t root = uf_find(parent, p);
    const double kd = ceil(wmax[p] * dt / theta_s);
    if (kd > 1e6) {
      free(parent); free(deg); free(wmax); free(scratch); free(order); free(kc);
      free(nb_j); free(fill);
      return -2;
    }
    const int64_t k = kd < 1.0 ? 1 : (int64_t)kd;
    if (k > kc[root]) kc[root] = k;
  }
  for (int64_t p = 0; p < n; p++)
    if (kc[p] > kmx) kmx = kc[p];
  if (n_pairs) *n_pairs = pairs;
  if (k_max) *k_max = kmx;
  /* the bodies of each cluster, grouped (order[] lists cluster members by
     root; a cluster is the run of equal roots) */
  int64_t cnt = 0;
  for (int64_t root = 0; root < n; root++) {
    if (kc[root] == 0) continue;
    for (int64_t p = 0; p < n; p++)
      if (deg[p + 1] > deg[p] && uf_find(parent, p) == root) order[cnt++] = p;
  }
  double *r[3] = {x, y, z}, *v[3] = {vx, vy, vz}, *a[3] = {ax, ay, az};
  double *an[3] = {anx, any, anz}, *f[3] = {fx, fy, fz};
  /* F = A_far: Eq. 1 for bodies in no cluster, the direct far sum for the rest */
  oracle_accel(n, G, x, y, z, m, ax, ay, az);
  for (int c = 0; c < 3; c++)
    for (int64_t p = 0; p < n; p++) f[c][p] = a[c][p];
  far_accel(n, G, x, y, z, m, order, cnt, deg, nb_j, fx, fy, fz);
  const double hd = 0.5 * dt;
  for (int64_t step = 0; step < n_steps; step++) {
    for (int c = 0; c < 3; c++) /* v <- v + dt/2 A_far(r) */
      for (int64_t p = 0; p < n; p++) v[c][p] = v[c][p] + hd * f[c][p];
    for (int c = 0; c < 3; c++) /* bodies in no cluster drift a full step */
      for (int64_t p = 0; p < n; p++)
        if (deg[p + 1] == deg[p]) r[c][p] = r[c][p] + dt * v[c][p];
    for (int64_t i0 = 0; i0 < cnt;) { /* each cluster: k sub-steps */
      const int64_t root = uf_find(parent, order[i0]);
      int64_t i1 = i0;
      while (i1 < cnt && uf_find(parent, order[i1]) == root) i1++;
      const int64_t k = kc[root];
      const double h = dt / (double)k, hh = 0.5 * h;
      for (int64_t sub = 0; sub < k; sub++) {
        near_accel(G, x, y, z, m, order + i0, i1 - i0, deg, nb_j, anx, any, anz);
        for (int64_t q = i0; q < i1; q++) {
          const int64_t p = order[q];
          for (int c = 0; c < 3; c++) {
            v[c][p] = v[c][p] + hh * an[c][p];
            r[c][p] = r[c][p] + h * v[c][p];
          }
        }
        near_accel(G, x, y, z, m, order + i0, i1 - i0, deg, nb_j, anx, any, anz);
        for (int64_t q = i0; q < i1; q++) {
          const int64_t p = order[q];
          for (int c = 0; c < 3; c++) v[c][p] = v[c][p] + hh * an[c][p];
        }
      }
      i0 = i1;
    }
    oracle_accel(n, G, x, y, z, m, ax, ay, az); /* Eq. 1 at the new r */
    for (int c = 0; c < 3; c++)
      for (int64_t p = 0; p < n; p++) f[c][p] = a[c][p];
    far_accel(n, G, x, y, z, m, order, cnt, deg, nb_j, fx, fy, fz);
    for (int c = 0; c < 3; c++) /* v <- v + dt/2 A_far(r) */
      for (int64_t p = 0; p < n; p++) v[c][p] = v[c][p] + hd * f[c][p];
  }
  free(parent); free(deg); free(wmax); free(scratch); free(order); free(kc);
  free(nb_j); free(fill);
  return 0;
}

/* 1 when built with OpenMP, else 0; and the thread count it would use. */
int oracle_openmp_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 0;
#endif
}
