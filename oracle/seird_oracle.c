/*
 * seird_oracle.c -- plain, slow, FP64 CPU oracle for the SEIRD reaction-diffusion
 * schemes of De Rosis, "A distribution-free lattice Boltzmann method for
 * compartmental reaction-diffusion systems with application to epidemic modelling"
 * (arXiv 2603.19789).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls
 * this file; only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header, table or constant with the CUDA path.
 *
 * Every routine takes the paper's steps in the paper's order, in double precision,
 * with no blocking, fusion or reordering beyond what the equations state.  OpenMP
 * only splits independent rows of one Jacobi sweep across host threads; the value
 * computed for each cell does not depend on the thread count.
 *
 * Storage: a state is 5 planes (S, E, I, R, D), each ny rows of nx cells, x fastest:
 *   state[c*ny*nx + y*nx + x].
 * Boundary codes: 0 = periodic, 1 = no-flux (homogeneous Neumann, Sec. II.C
 * "Mass conservation").  The cell-centred mirror reading of no-flux is used: a
 * neighbour outside the domain takes the value of the boundary cell itself.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

/* D2Q5 lattice, Sec. II.B: link vectors c_i and weights w_i; c_s^2 = 1/3. */
static const int CX[5] = {0, 1, 0, -1, 0};
static const int CY[5] = {0, 0, 1, 0, -1};
static const double W[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
static const int OPP[5] = {0, 3, 4, 1, 2};

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Relaxation time from a physical diffusivity, Eq. (diffusivity) with
 * c_s^2 = 1/3 in lattice units: d dt/dx^2 = (tau - 1/2)/3. */
double oracle_tau_from_d(double d, double dx, double dt) {
  double d_lattice = d * dt / (dx * dx);
  return 3.0 * d_lattice + 0.5;
}

/* Map an index that left the domain by one link back into it. */
static inline i64 wrap_or_clamp(i64 i, i64 n, int bc) {
  if (i >= 0 && i < n) return i;
  if (bc == 0) return (i < 0) ? i + n : i - n; /* periodic */
  return (i < 0) ? 0 : n - 1;                   /* mirror: the boundary cell itself */
}

static inline double val(const double* plane, i64 nx, i64 ny, int bc, i64 x, i64 y) {
  return plane[wrap_or_clamp(y, ny, bc) * nx + wrap_or_clamp(x, nx, bc)];
}

/* SEIRD reaction sources, Eq. (sources), and the deceased rate of Eq. (rhoD).
 * rates = {beta, alpha, gamma, phi} in the notation of Table I.
 * The force of infection uses the contact-eligible population N_c = S+E+I+R.
 * When N_c == 0 (all four mobile compartments empty) the force is taken as 0,
 * a case the paper leaves open. */
static void seird_sources(const double rates[4], double S, double E, double I, double R,
                          double psi[5]) {
  const double beta = rates[0], alpha = rates[1], gamma = rates[2], phi = rates[3];
  double Nc = S + E + I + R;
  double F = (Nc != 0.0) ? (beta * S) * I / Nc : 0.0;
  psi[0] = -F;                          /* S */
  psi[1] = F - alpha * E;               /* E */
  psi[2] = alpha * E - gamma * I;       /* I */
  psi[3] = (1.0 - phi) * gamma * I;     /* R */
  psi[4] = phi * gamma * I;             /* D, Eq. (rhoD) */
}

/*
 * One SSLBM step, Sec. II.C.  For each mobile compartment C in {S,E,I,R}:
 *   rho_f = sum_i w_i rho(x + c_i, t)            Eq. (rhof)
 *   rho_b = sum_i w_i rho(x - c_i, t)            Eq. (rhob)
 *   rho_c = rho(x, t)                             Eq. (rhoc)
 *   rho(x, t+dt) = rho_b + (tau^C - 1)(rho_f - 2 rho_c + rho_b) + Psi^C(x,t) dt
 *                                                 Eq. (sslbm_final_clean)
 * and for the deceased, the explicit update of the ODE Eq. (rhoD):
 *   D(x, t+dt) = D(x, t) + phi gamma I(x, t) dt.
 * All right-hand sides use time level t (Jacobi); `in` and `out` must differ.
 */
void oracle_sslbm_step(i64 nx, i64 ny, int bc, const double tau[4], const double rates[4],
                       double dt, const double* in, double* out) {
  const i64 M = nx * ny;
#pragma omp parallel for schedule(static)
  for (i64 y = 0; y < ny; ++y) {
    for (i64 x = 0; x < nx; ++x) {
      const i64 k = y * nx + x;
      double psi[5];
      seird_sources(rates, in[0 * M + k], in[1 * M + k], in[2 * M + k], in[3 * M + k], psi);
      for (int c = 0; c < 4; ++c) {
        const double* p = in + c * M;
        double rho_f = 0.0, rho_b = 0.0;
        for (int i = 0; i < 5; ++i) {
          rho_f += W[i] * val(p, nx, ny, bc, x + CX[i], y + CY[i]);
          rho_b += W[i] * val(p, nx, ny, bc, x - CX[i], y - CY[i]);
        }
        const double rho_c = p[k];
        out[c * M + k] = rho_b + (tau[c] - 1.0) * (rho_f - 2.0 * rho_c + rho_b) + psi[c] * dt;
      }
      out[4 * M + k] = in[4 * M + k] + psi[4] * dt;
    }
  }
}

/*
 * The SSLBM on the D2Q9 lattice (Sec. II.C, isotropy discussion): the same update,
 * Eq. (sslbm_final_clean), with rho_f and rho_b summed over the nine velocities
 * c_0 = (0,0), c_1..4 = (+-1,0),(0,+-1), c_5..8 = (+-1,+-1), weights 4/9, 1/9, 1/36, and
 * tau = 3 d dt / dx^2 + 1/2 (c_s^2 = 1/3 as on D2Q5).  Boundaries: periodic wrap per
 * coordinate; no-flux as halfway bounce-back, a link that leaves the domain sees the
 * cell's own value (on axis links this is the D2Q5 mirror; on diagonal links it keeps the
 * discrete population exactly conserved, which a per-coordinate mirror does not).
 */
static const int CX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W9[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static inline double val9(const double* plane, i64 nx, i64 ny, int bc, i64 x0, i64 y0, i64 x, i64 y) {
  if (bc == 0) return plane[wrap_or_clamp(y, ny, 0) * nx + wrap_or_clamp(x, nx, 0)];
  if (x < 0 || x >= nx || y < 0 || y >= ny) return plane[y0 * nx + x0];
  return plane[y * nx + x];
}

void oracle_sslbm9_step(i64 nx, i64 ny, int bc, const double tau[4], const double rates[4],
                        double dt, const double* in, double* out) {
  const i64 M = nx * ny;
#pragma omp parallel for schedule(static)
  for (i64 y = 0; y < ny; ++y) {
    for (i64 x = 0; x < nx; ++x) {
      const i64 k = y * nx + x;
      double psi[5];
      seird_sources(rates, in[0 * M + k], in[1 * M + k], in[2 * M + k], in[3 * M + k], psi);
      for (int c = 0; c < 4; ++c) {
        const double* p = in + c * M;
        double rho_f = 0.0, rho_b = 0.0;
        for (int i = 0; i < 9; ++i) {
          rho_f += W9[i] * val9(p, nx, ny, bc, x, y, x + CX9[i], y + CY9[i]);
          rho_b += W9[i] * val9(p, nx, ny, bc, x, y, x - CX9[i], y - CY9[i]);
        }
        const double rho_c = p[k];
        out[c * M + k] = rho_b + (tau[c] - 1.0) * (rho_f - 2.0 * rho_c + rho_b) + psi[c] * dt;
      }
      out[4 * M + k] = in[4 * M + k] + psi[4] * dt;
    }
  }
}

void oracle_sslbm9_run(i64 nx, i64 ny, int bc, const double tau[4], const double rates[4],
                       double dt, i64 nsteps, double* state, double* scratch) {
  const i64 n = 5 * nx * ny;
  double* a = state;
  double* b = scratch;
  for (i64 s = 0; s < nsteps; ++s) {
    oracle_sslbm9_step(nx, ny, bc, tau, rates, dt, a, b);
    double* t = a;
    a = b;
    b = t;
  }
  if (a != state) memcpy(state, a, (size_t)n * sizeof(double));
}

/*
 * The two-pass simplified LBM (SLBM) of Sec. II.C, Eqs. (SLBM1, SLBM2), on D2Q5:
 *   predictor  rho*(x)   = sum_i w_i rho(x - c_i, t)
 *   corrector  rho(x, t+dt) = rho*(x) + (tau - 1)(sum_i w_i rho*(x + c_i) - rho(x, t))
 *                             + Psi(x, t) dt
 * for C in {S, E, I, R}; D takes the explicit update of Eq. (rhoD).  Neighbours follow the
 * same rule as the SSLBM (periodic wrap or the cell-centred mirror).  `pred` is a scratch
 * of 4 planes.
 */
void oracle_slbm_step(i64 nx, i64 ny, int bc, const double tau[4], const double rates[4], double dt,
                      const double* in, double* pred, double* out) {
  const i64 M = nx * ny;
#pragma omp parallel for schedule(static)
  for (i64 y = 0; y < ny; ++y)
    for (i64 x = 0; x < nx; ++x)
      for (int c = 0; c < 4; ++c) {
        const double* p = in + c * M;
        double r = 0.0;
        for (int i = 0; i < 5; ++i) r += W[i] * val(p, nx, ny, bc, x - CX[i], y - CY[i]);
        pred[c * M + y * nx + x] = r;
      }
#pragma omp parallel for schedule(static)
  for (i64 y = 0; y < ny; ++y)
    for (i64 x = 0; x < nx; ++x) {
      const i64 k = y * nx + x;
      double psi[5];
      seird_sources(rates, in[0 * M + k], in[1 * M + k], in[2 * M + k], in[3 * M + k], psi);
      for (int c = 0; c < 4; ++c) {
        const double* q = pred + c * M;
        double s = 0.0;
        for (int i = 0; i < 5; ++i) s += W[i] * val(q, nx, ny, bc, x + CX[i], y + CY[i]);
        out[c * M + k] = q[k] + (tau[c] - 1.0) * (s - in[c * M + k]) + psi[c] * dt;
      }
      out[4 * M + k] = in[4 * M + k] + psi[4] * dt;
    }
}

void oracle_slbm_run(i64 nx, i64 ny, int bc, const double tau[4], const double rates[4], double dt,
                     i64 nsteps, double* state, double* scratch) {
  const i64 n = 5 * nx * ny;
  double* pred = (double*)malloc((size_t)(4 * nx * ny) * sizeof(double));
  double* a = state;
  double* b = scratch;
  for (i64 s = 0; s < nsteps; ++s) {
    oracle_slbm_step(nx, ny, bc, tau, rates, dt, a, pred, b);
    double* t = a;
    a = b;
    b = t;
  }
  if (a != state) memcpy(state, a, (size_t)n * sizeof(double));
  free(pred);
}

/*
 * The SSLBM with spatially varying, axis-anisotropic diffusion: the extension Sec. IV lists
 * among the directions for future work.  The paper gives no discretisation for it; this is
 * the reading the library uses.  The D2Q5 update in its link (flux) form,
 *   rho(x, t+dt) = rho_c + sum_{i=1..4} D_i(x) (rho(x + c_i, t) - rho_c) + Psi(x, t) dt,
 *   D_i(x) = d_lattice^C (k_a(x) + k_a(x + c_i)) / 2,
 * with a = x on the links c_1, c_3 and a = y on c_2, c_4, d_lattice^C = (tau^C - 1/2) / 3,
 * and per-cell scale fields kx, ky >= 0.  With kx = ky = 1 this is Eq. (sslbm_final_clean)
 * on D2Q5, where rho_f = rho_b and rho_b + (tau - 1)(rho_f - 2 rho_c + rho_b)
 * = rho_c + d_lattice sum_i (rho(x + c_i) - rho_c).  Both cells of a link use the same
 * coefficient, so what one gains the other loses and the population total is conserved as
 * in Sec. II.C.  Neighbours (of rho and of the scale fields) follow oracle_sslbm_step: the
 * periodic wrap, or the boundary cell itself, whose difference is zero (no flux through a
 * wall).  kx, ky: ny*nx values each, x fastest.  D takes the update of Eq. (rhoD).
 */
void oracle_sslbm_vard_step(i64 nx, i64 ny, int bc, const double tau[4], const double rates[4], double dt,
                            const double* kx, const double* ky, const double* in, double* out) {
  const i64 M = nx * ny;
#pragma omp parallel for schedule(static)
  for (i64 y = 0; y < ny; ++y) {
    for (i64 x = 0; x < nx; ++x) {
      const i64 k = y * nx + x;
      double psi[5];
      seird_sources(rates, in[0 * M + k], in[1 * M + k], in[2 * M + k], in[3 * M + k], psi);
      for (int c = 0; c < 4; ++c) {
        const double* p = in + c * M;
        const double d_lattice = (tau[c] - 0.5) / 3.0;
        const double rho_c = p[k];
        double flux = 0.0;
        for (int i = 1; i < 5; ++i) {
          const double* kap = CX[i] != 0 ? kx : ky;
          const double k_link = 0.5 * (kap[k] + val(kap, nx, ny, bc, x + CX[i], y + CY[i]));
          flux += k_link * (val(p, nx, ny, bc, x + CX[i], y + CY[i]) - rho_c);
        }
        out[c * M + k] = rho_c + d_lattice * flux + psi[c] * dt;
      }
      out[4 * M + k] = in[4 * M + k] + psi[4] * dt;
    }
  }
}

void oracle_sslbm_vard_run(i64 nx, i64 ny, int bc, const double tau[4], const double rates[4], double dt,
                           const double* kx, const double* ky, i64 nsteps, double* state, double* scratch) {
  const i64 n = 5 * nx * ny;
  double* a = state;
  double* b = scratch;
  for (i64 s = 0; s < nsteps; ++s) {
    oracle_sslbm_vard_step(nx, ny, bc, tau, rates, dt, kx, ky, a, b);
    double* t = a;
    a = b;
    b = t;
  }
  if (a != state) memcpy(state, a, (size_t)n * sizeof(double));
}

/* nsteps SSLBM steps; `state` holds the input and receives the result,
 * `scratch` is a second state-sized buffer. */
void oracle_sslbm_run(i64 nx, i64 ny, int bc, const double tau[4], const double rates[4],
                      double dt, i64 nsteps, double* state, double* scratch) {
  const i64 n = 5 * nx * ny;
  double* a = state;
  double* b = scratch;
  for (i64 s = 0; s < nsteps; ++s) {
    oracle_sslbm_step(nx, ny, bc, tau, rates, dt, a, b);
    double* t = a;
    a = b;
    b = t;
  }
  if (a != state) memcpy(state, a, (size_t)n * sizeof(double));
}

/*
 * BGK lattice Boltzmann, Sec. II.B.  PDFs f[c][i][y][x] for the four mobile
 * compartments c and the five D2Q5 directions i; the deceased density is carried
 * as a plain field (it does not diffuse, Sec. II.B storage count).
 *
 * Initialisation (left open by the paper): the equilibrium f_i = w_i rho(x, 0).
 */
void oracle_bgk_init(i64 nx, i64 ny, const double* state, double* f) {
  const i64 M = nx * ny;
  for (int c = 0; c < 4; ++c)
    for (int i = 0; i < 5; ++i)
      for (i64 k = 0; k < M; ++k) f[(c * 5 + i) * M + k] = W[i] * state[c * M + k];
}

/* rho^C = sum_i f_i^C (Sec. II.B), written into planes 0..3 of `state`. */
void oracle_bgk_density(i64 nx, i64 ny, const double* f, double* state) {
  const i64 M = nx * ny;
  for (int c = 0; c < 4; ++c)
    for (i64 k = 0; k < M; ++k) {
      double rho = 0.0;
      for (int i = 0; i < 5; ++i) rho += f[(c * 5 + i) * M + k];
      state[c * M + k] = rho;
    }
}

/*
 * One BGK step, Eq. (pdf):
 *   f_i(x + c_i, t+dt) = f_i + (w_i rho - f_i)/tau + w_i Psi dt,
 * with rho = sum_i f_i and Psi from Eq. (sources) at (x, t), and the deceased
 * updated by Eq. (rhoD).  Written in pull form: the population i arriving at x
 * left x - c_i.  For no-flux walls, halfway bounce-back: when x - c_i lies outside
 * the domain, the arriving population is the post-collision population of the
 * opposite direction at x itself (it hit the wall face and came back).
 */
void oracle_bgk_step(i64 nx, i64 ny, int bc, const double tau[4], const double rates[4],
                     double dt, const double* f_in, const double* D_in, double* f_out,
                     double* D_out) {
  const i64 M = nx * ny;
  /* post-collision populations, computed cell by cell */
  double* post = (double*)malloc((size_t)(20 * M) * sizeof(double));
#pragma omp parallel for schedule(static)
  for (i64 k = 0; k < M; ++k) {
    double rho[4];
    for (int c = 0; c < 4; ++c) {
      double r = 0.0;
      for (int i = 0; i < 5; ++i) r += f_in[(c * 5 + i) * M + k];
      rho[c] = r;
    }
    double psi[5];
    seird_sources(rates, rho[0], rho[1], rho[2], rho[3], psi);
    for (int c = 0; c < 4; ++c)
      for (int i = 0; i < 5; ++i) {
        const double fi = f_in[(c * 5 + i) * M + k];
        post[(c * 5 + i) * M + k] = fi + (W[i] * rho[c] - fi) / tau[c] + W[i] * psi[c] * dt;
      }
    D_out[k] = D_in[k] + psi[4] * dt;
  }
#pragma omp parallel for schedule(static)
  for (i64 y = 0; y < ny; ++y)
    for (i64 x = 0; x < nx; ++x) {
      const i64 k = y * nx + x;
      for (int c = 0; c < 4; ++c)
        for (int i = 0; i < 5; ++i) {
          i64 xs = x - CX[i], ys = y - CY[i];
          double v;
          if (xs >= 0 && xs < nx && ys >= 0 && ys < ny) {
            v = post[(c * 5 + i) * M + ys * nx + xs];
          } else if (bc == 0) {
            xs = wrap_or_clamp(xs, nx, 0);
            ys = wrap_or_clamp(ys, ny, 0);
            v = post[(c * 5 + i) * M + ys * nx + xs];
          } else {
            v = post[(c * 5 + OPP[i]) * M + k];
          }
          f_out[(c * 5 + i) * M + k] = v;
        }
    }
  free(post);
}

void oracle_bgk_run(i64 nx, i64 ny, int bc, const double tau[4], const double rates[4], double dt,
                    i64 nsteps, double* f, double* D) {
  const i64 M = nx * ny;
  double* f2 = (double*)malloc((size_t)(20 * M) * sizeof(double));
  double* D2 = (double*)malloc((size_t)M * sizeof(double));
  double *fa = f, *fb = f2, *Da = D, *Db = D2;
  for (i64 s = 0; s < nsteps; ++s) {
    oracle_bgk_step(nx, ny, bc, tau, rates, dt, fa, Da, fb, Db);
    double* t = fa; fa = fb; fb = t;
    t = Da; Da = Db; Db = t;
  }
  if (fa != f) memcpy(f, fa, (size_t)(20 * M) * sizeof(double));
  if (Da != D) memcpy(D, Da, (size_t)M * sizeof(double));
  free(f2);
  free(D2);
}

/*
 * Fourth-order finite-difference reference, Sec. III: classical RK4 in time and
 * the fourth-order centred Laplacian in space,
 *   L4 u = sum over axes of (-u[-2] + 16 u[-1] - 30 u[0] + 16 u[+1] - u[+2]) / (12 dx^2),
 * with the reactions evaluated explicitly at every stage.
 * Right-hand side, Eqs. (EqSEIRD_S..D): d/dt C = Psi^C + d^C L4 C for C in {S,E,I,R},
 * d/dt D = phi gamma I.  Ghost cells: periodic wrap, or (no-flux) an even
 * reflection about the boundary face: u[-1] = u[0], u[-2] = u[1].
 */
static inline i64 ghost2(i64 i, i64 n, int bc) {
  if (i >= 0 && i < n) return i;
  if (bc == 0) {
    i64 r = i % n;
    return r < 0 ? r + n : r;
  }
  if (i < 0) i = -1 - i;
  if (i >= n) i = 2 * n - 1 - i;
  if (i < 0) i = 0;       /* grids narrower than the stencil */
  if (i >= n) i = n - 1;
  return i;
}

static void fd4_rhs(i64 nx, i64 ny, int bc, const double d[4], const double rates[4], double dx,
                    const double* u, double* rhs) {
  const i64 M = nx * ny;
  const double inv = 1.0 / (12.0 * dx * dx);
#pragma omp parallel for schedule(static)
  for (i64 y = 0; y < ny; ++y)
    for (i64 x = 0; x < nx; ++x) {
      const i64 k = y * nx + x;
      double psi[5];
      seird_sources(rates, u[k], u[M + k], u[2 * M + k], u[3 * M + k], psi);
      for (int c = 0; c < 4; ++c) {
        const double* p = u + c * M;
        const double u0 = p[k];
        double lx = -p[y * nx + ghost2(x - 2, nx, bc)] + 16.0 * p[y * nx + ghost2(x - 1, nx, bc)] -
                    30.0 * u0 + 16.0 * p[y * nx + ghost2(x + 1, nx, bc)] -
                    p[y * nx + ghost2(x + 2, nx, bc)];
        double ly = -p[ghost2(y - 2, ny, bc) * nx + x] + 16.0 * p[ghost2(y - 1, ny, bc) * nx + x] -
                    30.0 * u0 + 16.0 * p[ghost2(y + 1, ny, bc) * nx + x] -
                    p[ghost2(y + 2, ny, bc) * nx + x];
        rhs[c * M + k] = psi[c] + d[c] * (lx + ly) * inv;
      }
      rhs[4 * M + k] = psi[4];
    }
}

/*
 * Second-order counterpart for the cost comparison of Sec. IV (Table tab:timing, "FDM
 * 2nd"): the same classical RK4 with the second-order centred Laplacian
 *   L2 u = sum over axes of (u[-1] - 2 u[0] + u[+1]) / dx^2,
 * the same sources and the same ghost rule.
 */
static void fd2_rhs(i64 nx, i64 ny, int bc, const double d[4], const double rates[4], double dx,
                    const double* u, double* rhs) {
  const i64 M = nx * ny;
  const double inv = 1.0 / (dx * dx);
#pragma omp parallel for schedule(static)
  for (i64 y = 0; y < ny; ++y)
    for (i64 x = 0; x < nx; ++x) {
      const i64 k = y * nx + x;
      double psi[5];
      seird_sources(rates, u[k], u[M + k], u[2 * M + k], u[3 * M + k], psi);
      for (int c = 0; c < 4; ++c) {
        const double* p = u + c * M;
        const double u0 = p[k];
        double lx = p[y * nx + ghost2(x - 1, nx, bc)] - 2.0 * u0 + p[y * nx + ghost2(x + 1, nx, bc)];
        double ly = p[ghost2(y - 1, ny, bc) * nx + x] - 2.0 * u0 + p[ghost2(y + 1, ny, bc) * nx + x];
        rhs[c * M + k] = psi[c] + d[c] * (lx + ly) * inv;
      }
      rhs[4 * M + k] = psi[4];
    }
}

void oracle_fd2_rk4_run(i64 nx, i64 ny, int bc, const double d[4], const double rates[4],
                        double dx, double dt, i64 nsteps, double* state) {
  const i64 n = 5 * nx * ny;
  double* k1 = (double*)malloc((size_t)n * sizeof(double));
  double* k2 = (double*)malloc((size_t)n * sizeof(double));
  double* k3 = (double*)malloc((size_t)n * sizeof(double));
  double* k4 = (double*)malloc((size_t)n * sizeof(double));
  double* tmp = (double*)malloc((size_t)n * sizeof(double));
  for (i64 s = 0; s < nsteps; ++s) {
    fd2_rhs(nx, ny, bc, d, rates, dx, state, k1);
    for (i64 j = 0; j < n; ++j) tmp[j] = state[j] + 0.5 * dt * k1[j];
    fd2_rhs(nx, ny, bc, d, rates, dx, tmp, k2);
    for (i64 j = 0; j < n; ++j) tmp[j] = state[j] + 0.5 * dt * k2[j];
    fd2_rhs(nx, ny, bc, d, rates, dx, tmp, k3);
    for (i64 j = 0; j < n; ++j) tmp[j] = state[j] + dt * k3[j];
    fd2_rhs(nx, ny, bc, d, rates, dx, tmp, k4);
    for (i64 j = 0; j < n; ++j)
      state[j] += dt / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
  }
  free(k1); free(k2); free(k3); free(k4); free(tmp);
}

void oracle_fd4_rk4_run(i64 nx, i64 ny, int bc, const double d[4], const double rates[4],
                        double dx, double dt, i64 nsteps, double* state) {
  const i64 n = 5 * nx * ny;
  double* k1 = (double*)malloc((size_t)n * sizeof(double));
  double* k2 = (double*)malloc((size_t)n * sizeof(double));
  double* k3 = (double*)malloc((size_t)n * sizeof(double));
  double* k4 = (double*)malloc((size_t)n * sizeof(double));
  double* tmp = (double*)malloc((size_t)n * sizeof(double));
  for (i64 s = 0; s < nsteps; ++s) {
    fd4_rhs(nx, ny, bc, d, rates, dx, state, k1);
    for (i64 j = 0; j < n; ++j) tmp[j] = state[j] + 0.5 * dt * k1[j];
    fd4_rhs(nx, ny, bc, d, rates, dx, tmp, k2);
    for (i64 j = 0; j < n; ++j) tmp[j] = state[j] + 0.5 * dt * k2[j];
    fd4_rhs(nx, ny, bc, d, rates, dx, tmp, k3);
    for (i64 j = 0; j < n; ++j) tmp[j] = state[j] + dt * k3[j];
    fd4_rhs(nx, ny, bc, d, rates, dx, tmp, k4);
    for (i64 j = 0; j < n; ++j)
      state[j] += dt / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
  }
  free(k1); free(k2); free(k3); free(k4); free(tmp);
}

/* The spatially homogeneous SEIRD system (Eqs. EqSEIRD_S..D without diffusion),
 * integrated by classical RK4 with step dt.  y = {S, E, I, R, D}. */
void oracle_ode_rk4(const double rates[4], double dt, i64 nsteps, double y[5]) {
  double k1[5], k2[5], k3[5], k4[5], t[5];
  for (i64 s = 0; s < nsteps; ++s) {
    seird_sources(rates, y[0], y[1], y[2], y[3], k1);
    for (int j = 0; j < 5; ++j) t[j] = y[j] + 0.5 * dt * k1[j];
    seird_sources(rates, t[0], t[1], t[2], t[3], k2);
    for (int j = 0; j < 5; ++j) t[j] = y[j] + 0.5 * dt * k2[j];
    seird_sources(rates, t[0], t[1], t[2], t[3], k3);
    for (int j = 0; j < 5; ++j) t[j] = y[j] + dt * k3[j];
    seird_sources(rates, t[0], t[1], t[2], t[3], k4);
    for (int j = 0; j < 5; ++j) y[j] += dt / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
  }
}

/* Reaction sources at one point, exposed for tests of Eq. (sources). */
void oracle_sources(const double rates[4], const double rho[4], double psi[5]) {
  seird_sources(rates, rho[0], rho[1], rho[2], rho[3], psi);
}

/*
 * Diagnostics of Sec. II.C "Mass conservation": per-compartment totals
 * sum_x rho^C(x) (Neumaier-compensated, so the result is the exact sum to
 * within a few ulp) and the peak of the infected density.
 */
void oracle_diagnostics(i64 nx, i64 ny, const double* state, double totals[5], double* peak_I) {
  const i64 M = nx * ny;
  for (int c = 0; c < 5; ++c) {
    double s = 0.0, comp = 0.0;
    for (i64 k = 0; k < M; ++k) {
      const double v = state[c * M + k];
      const double t = s + v;
      if (fabs(s) >= fabs(v))
        comp += (s - t) + v;
      else
        comp += (v - t) + s;
      s = t;
    }
    totals[c] = s + comp;
  }
  double m = -INFINITY;
  for (i64 k = 0; k < M; ++k)
    if (state[2 * M + k] > m) m = state[2 * M + k];
  *peak_I = m;
}
