/*
 * fv_oracle.c -- plain, slow, FP64 CPU oracle for the batched finite-volume
 * patch update of arXiv 2302.09005 ("GPU Offloading in ExaHyPE Through C++
 * Standard Algorithms").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA library in
 * paper_2302_09005_gb300/csrc and neither includes the other.
 *
 * What it computes, and where the paper defines it:
 *   - Euler flux f^j(q) of the compressible Euler equations, Eq. 2 (Sec. 2),
 *     with the energy flux read as (E_t + p) j_j / rho (the printed formula
 *     lacks the factor j_j, without which it would not be a flux along j).
 *   - Maximum wave speed |u_j| + c, c = sqrt(gamma p / rho): the largest
 *     |eigenvalue| of the Euler flux Jacobian in direction j, Eq. 5.
 *     "Between Q_{i-1} and Q_i" is read as the maximum over the two states.
 *   - Rusanov face flux, Eq. 4:
 *       F_{i-1/2} = 1/2 [ f(Q_{i-1}) + f(Q_i) - a_{i-1/2} (Q_i - Q_{i-1}) ].
 *   - Explicit Euler finite-volume update, Eq. 3, summed over the 2d faces of
 *     the cell (Algorithm 1, step 7):
 *       Q_i^{n+1} = Q_i^n - dt/dx * sum_j (F_{i+1/2 e_j} - F_{i-1/2 e_j}).
 *   - Per-patch maximum eigenvalue (Algorithm 1, step 10): the largest a over
 *     the faces the update used.
 *   - Halo fill: the engine keeps the one-cell halo layer of every patch
 *     consistent with its neighbours (Sec. 2, "each patch is supplemented
 *     with a halo layer").
 *
 * Layout (shared convention, not shared code): patch i occupies the
 * elements [off[i], off[i] + (p+2h)^d * s) of the buffer.  Cells run x
 * fastest, then y, then z; the s unknowns of a cell are contiguous.
 * Interior cells have every coordinate in [h, h+p).
 *
 * Built with -O2 -ffp-contract=off: no fused multiply-add, every operation
 * rounded as written.  Single-threaded.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_BAD_ARG 1

enum { ORC_PDE_EULER = 0, ORC_PDE_ADVECTION = 1 };

/* ---------------------------------------------------------------------- */
/* Physics                                                                 */
/* ---------------------------------------------------------------------- */

/* Pressure of the ideal gas from the conserved state q = (rho, j_1..j_d, E):
 * p = (gamma - 1) (E - |j|^2 / (2 rho))   (equation of state behind Eq. 2). */
static double euler_pressure(const double *q, int d, double gamma) {
  double rho = q[0];
  double jj = 0.0;
  for (int k = 0; k < d; ++k) jj = jj + q[1 + k] * q[1 + k];
  return (gamma - 1.0) * (q[d + 1] - 0.5 * jj / rho);
}

/* Flux f^dir(q) of Eq. 2: (j_dir, j u_dir + p e_dir, (E + p) u_dir). */
void orc_euler_flux(const double *q, int d, int dir, double gamma, double *f) {
  double rho = q[0];
  double p = euler_pressure(q, d, gamma);
  double u = q[1 + dir] / rho;
  f[0] = q[1 + dir];
  for (int k = 0; k < d; ++k) f[1 + k] = q[1 + k] * u + (k == dir ? p : 0.0);
  f[d + 1] = (q[d + 1] + p) * u;
}

/* Largest |eigenvalue| of the flux Jacobian in direction dir: |u_dir| + c,
 * c = sqrt(gamma p / rho) (Eq. 5). */
double orc_euler_wave_speed(const double *q, int d, int dir, double gamma) {
  double rho = q[0];
  double p = euler_pressure(q, d, gamma);
  double u = q[1 + dir] / rho;
  double c = sqrt(gamma * p / rho);
  return fabs(u) + c;
}

/* Generic flux and wave speed: the Euler system, or (tests only) linear
 * advection f^dir(q) = adv[dir] q with wave speed |adv[dir]|, a PDE of the
 * class of Eq. 1 for which the Rusanov scheme is first-order upwind. */
static void pde_flux(int pde, const double *q, int d, int s, int dir, double gamma,
                     const double *adv, double *f, double *lam) {
  if (pde == ORC_PDE_ADVECTION) {
    for (int v = 0; v < s; ++v) f[v] = adv[dir] * q[v];
    *lam = fabs(adv[dir]);
  } else {
    orc_euler_flux(q, d, dir, gamma, f);
    *lam = orc_euler_wave_speed(q, d, dir, gamma);
  }
}

/* Rusanov flux of Eq. 4 between left state qL (= Q_{i-1}) and right state
 * qR (= Q_i) in direction dir.  a = max(lambda_L, lambda_R) (Eq. 5). */
static void rusanov(int pde, const double *qL, const double *qR, int d, int s, int dir,
                    double gamma, const double *adv, double *F, double *a_out) {
  double fL[8], fR[8], lamL, lamR;
  pde_flux(pde, qL, d, s, dir, gamma, adv, fL, &lamL);
  pde_flux(pde, qR, d, s, dir, gamma, adv, fR, &lamR);
  double a = lamL > lamR ? lamL : lamR;
  for (int v = 0; v < s; ++v) F[v] = 0.5 * ((fL[v] + fR[v]) - a * (qR[v] - qL[v]));
  *a_out = a;
}

void orc_rusanov_flux(const double *qL, const double *qR, int d, int dir, double gamma,
                      double *F, double *a_out) {
  rusanov(ORC_PDE_EULER, qL, qR, d, d + 2, dir, gamma, NULL, F, a_out);
}

/* ---------------------------------------------------------------------- */
/* Patch indexing                                                          */
/* ---------------------------------------------------------------------- */

/* Element index of unknown 0 of cell (c[0], c[1], c[2]) in a patch whose
 * halo-inclusive edge length is n. */
static int64_t cell_index(const int *c, int d, int n) {
  int64_t idx = 0;
  for (int k = d - 1; k >= 0; --k) idx = idx * n + c[k];
  return idx;
}

static int check_patch_args(const int64_t *off, const int32_t *sizes, int64_t n, int d, int s,
                            int h) {
  if (n < 0 || d < 1 || d > 3 || s < 1 || s > 8 || h < 1) return ORC_BAD_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (sizes[i] < 1 || off[i] < 0) return ORC_BAD_ARG;
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Patch update: Eq. 3 with the face fluxes of Eq. 4                       */
/* ---------------------------------------------------------------------- */

/* One explicit Euler step of every patch of the batch (Algorithm 1 with the
 * outer loop over patches).  Interior cells of out are written; the halo of
 * out is left untouched.  lam_patch (nullable) receives, per patch, the
 * largest a over the faces used (Algorithm 1, step 10). */
int orc_patch_update_pde(int pde, const double *adv, const double *in, double *out,
                         const int64_t *off, const int32_t *sizes, int64_t n, int d, int s,
                         int h, double gamma, double dx, double dt, double *lam_patch) {
  if (check_patch_args(off, sizes, n, d, s, h) != ORC_OK) return ORC_BAD_ARG;
  if (pde == ORC_PDE_EULER && s != d + 2) return ORC_BAD_ARG;
  double r = dt / dx;
  for (int64_t i = 0; i < n; ++i) {
    int p = sizes[i];
    int ne = p + 2 * h;
    const double *Q = in + off[i];
    double *Qo = out + off[i];
    double lam_max = 0.0;
    int ncell = 1;
    for (int k = 0; k < d; ++k) ncell *= p;
    for (int t = 0; t < ncell; ++t) {
      /* interior cell coordinates, x fastest */
      int c[3] = {0, 0, 0};
      int rem = t;
      for (int k = 0; k < d; ++k) {
        c[k] = h + rem % p;
        rem /= p;
      }
      const double *qc = Q + cell_index(c, d, ne) * s;
      double acc[8];
      for (int v = 0; v < s; ++v) acc[v] = 0.0;
      for (int k = 0; k < d; ++k) {
        int cm[3] = {c[0], c[1], c[2]}, cp[3] = {c[0], c[1], c[2]};
        cm[k] -= 1;
        cp[k] += 1;
        const double *qm = Q + cell_index(cm, d, ne) * s;
        const double *qp = Q + cell_index(cp, d, ne) * s;
        double Fm[8], Fp[8], am, ap;
        rusanov(pde, qm, qc, d, s, k, gamma, adv, Fm, &am); /* face i-1/2 */
        rusanov(pde, qc, qp, d, s, k, gamma, adv, Fp, &ap); /* face i+1/2 */
        for (int v = 0; v < s; ++v) acc[v] = acc[v] + (Fp[v] - Fm[v]);
        if (am > lam_max) lam_max = am;
        if (ap > lam_max) lam_max = ap;
      }
      double *qo = Qo + cell_index(c, d, ne) * s;
      for (int v = 0; v < s; ++v) qo[v] = qc[v] - r * acc[v];
    }
    if (lam_patch) lam_patch[i] = lam_max;
  }
  return ORC_OK;
}

int orc_patch_update(const double *in, double *out, const int64_t *off, const int32_t *sizes,
                     int64_t n, int d, int h, double gamma, double dx, double dt,
                     double *lam_patch) {
  return orc_patch_update_pde(ORC_PDE_EULER, NULL, in, out, off, sizes, n, d, d + 2, h, gamma,
                              dx, dt, lam_patch);
}

/* ---------------------------------------------------------------------- */
/* Maximum eigenvalue per patch and over the batch, and the CFL time step  */
/* ---------------------------------------------------------------------- */

/* Per patch: the largest a over the faces that bound interior cells (the
 * same set of faces the update uses), i.e. the patch maximum eigenvalue of
 * Algorithm 1, step 10, evaluated on the given state.  lam_global receives
 * the maximum over the batch (0 for an empty batch). */
int orc_max_eigenvalue(const double *q, const int64_t *off, const int32_t *sizes, int64_t n,
                       int d, int h, double gamma, double *lam_patch, double *lam_global) {
  int s = d + 2;
  if (check_patch_args(off, sizes, n, d, s, h) != ORC_OK) return ORC_BAD_ARG;
  double gmax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    int p = sizes[i];
    int ne = p + 2 * h;
    const double *Q = q + off[i];
    double lam_max = 0.0;
    for (int k = 0; k < d; ++k) {
      /* faces normal to k: left cell coordinate along k in [h-1, h+p-1],
       * other coordinates interior. */
      int nf = p + 1;
      for (int k2 = 0; k2 < d; ++k2)
        if (k2 != k) nf *= p;
      for (int t = 0; t < nf; ++t) {
        int c[3] = {0, 0, 0};
        int rem = t;
        for (int k2 = 0; k2 < d; ++k2) {
          int len = (k2 == k) ? p + 1 : p;
          c[k2] = (k2 == k ? h - 1 : h) + rem % len;
          rem /= len;
        }
        int cr[3] = {c[0], c[1], c[2]};
        cr[k] += 1;
        double lamL = orc_euler_wave_speed(Q + cell_index(c, d, ne) * s, d, k, gamma);
        double lamR = orc_euler_wave_speed(Q + cell_index(cr, d, ne) * s, d, k, gamma);
        double a = lamL > lamR ? lamL : lamR;
        if (a > lam_max) lam_max = a;
      }
    }
    if (lam_patch) lam_patch[i] = lam_max;
    if (lam_max > gmax) gmax = lam_max;
  }
  if (lam_global) *lam_global = gmax;
  return ORC_OK;
}

/* CFL time step: dt = cfl * dx / (d * lambda_max).  The factor d keeps the
 * unsplit d-dimensional update stable (a reading: the paper does not define
 * the CFL condition). */
double orc_cfl_dt(double lam_max, double cfl, double dx, int d) {
  return cfl * dx / ((double)d * lam_max);
}

/* ---------------------------------------------------------------------- */
/* Halo fill                                                               */
/* ---------------------------------------------------------------------- */

/* Fills the face halo layers of every patch (edge and corner halo cells are
 * not touched).  nbr has 2d entries per patch in the order -x,+x,-y,+y,-z,+z:
 *   nbr >= 0 : the neighbouring patch (same p); its interior layers next to
 *              the shared face are copied (a patch that is its own neighbour
 *              is periodic);
 *   nbr == -1: outflow, the halo repeats the nearest interior cell;
 *   nbr == -2: reflecting wall, the mirror image of the interior with the
 *              normal momentum component (unknown 1+k) negated.
 * Reads only interior cells and writes only halo cells, so it runs in place. */
int orc_halo_fill(double *q, const int64_t *off, const int32_t *sizes, const int32_t *nbr,
                  int64_t n, int d, int s, int h) {
  if (check_patch_args(off, sizes, n, d, s, h) != ORC_OK) return ORC_BAD_ARG;
  for (int64_t i = 0; i < n; ++i) {
    int p = sizes[i];
    if (p < h) return ORC_BAD_ARG;
    int ne = p + 2 * h;
    double *Q = q + off[i];
    for (int k = 0; k < d; ++k) {
      for (int side = 0; side < 2; ++side) {
        int32_t nb = nbr[i * 2 * d + 2 * k + side];
        if (nb >= n || nb < -2) return ORC_BAD_ARG;
        if (nb >= 0 && sizes[nb] != p) return ORC_BAD_ARG;
        const double *S = nb >= 0 ? q + off[nb] : Q;
        int ncell = h;
        for (int k2 = 0; k2 < d; ++k2)
          if (k2 != k) ncell *= p;
        for (int t = 0; t < ncell; ++t) {
          int c[3] = {0, 0, 0};
          int rem = t;
          for (int k2 = 0; k2 < d; ++k2) {
            int len = (k2 == k) ? h : p;
            c[k2] = (k2 == k ? 0 : h) + rem % len;
            rem /= len;
          }
          int l = c[k]; /* halo layer: 0 is the layer on the interior */
          int dst = side == 0 ? h - 1 - l : h + p + l;
          int src;
          if (nb >= 0)
            src = side == 0 ? dst + p : dst - p;
          else if (nb == -1)
            src = side == 0 ? h : h + p - 1;
          else
            src = side == 0 ? h + l : h + p - 1 - l;
          int cd[3] = {c[0], c[1], c[2]}, cs[3] = {c[0], c[1], c[2]};
          cd[k] = dst;
          cs[k] = src;
          double *qd = Q + cell_index(cd, d, ne) * s;
          const double *qs = S + cell_index(cs, d, ne) * s;
          for (int v = 0; v < s; ++v) qd[v] = qs[v];
          if (nb == -2 && 1 + k < s) qd[1 + k] = -qs[1 + k];
        }
      }
    }
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Conserved totals                                                        */
/* ---------------------------------------------------------------------- */

/* Per-patch sums of every unknown over the interior cells, cells visited x
 * fastest.  sums has n * s entries. */
int orc_patch_sums(const double *q, const int64_t *off, const int32_t *sizes, int64_t n, int d,
                   int s, int h, double *sums) {
  if (check_patch_args(off, sizes, n, d, s, h) != ORC_OK) return ORC_BAD_ARG;
  for (int64_t i = 0; i < n; ++i) {
    int p = sizes[i];
    int ne = p + 2 * h;
    const double *Q = q + off[i];
    double acc[8];
    for (int v = 0; v < s; ++v) acc[v] = 0.0;
    int ncell = 1;
    for (int k = 0; k < d; ++k) ncell *= p;
    for (int t = 0; t < ncell; ++t) {
      int c[3] = {0, 0, 0};
      int rem = t;
      for (int k = 0; k < d; ++k) {
        c[k] = h + rem % p;
        rem /= p;
      }
      const double *qc = Q + cell_index(c, d, ne) * s;
      for (int v = 0; v < s; ++v) acc[v] = acc[v] + qc[v];
    }
    for (int v = 0; v < s; ++v) sums[i * s + v] = acc[v];
  }
  return ORC_OK;
}
