/*
 * oracle.c -- plain FP64 CPU reference of the explicit finite-difference
 * acoustic solver of "simwave" (arXiv 2201.05278).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into oracle/liboracle.so and
 * is called from tests/, from __graft_entry__.smoke() and from the CPU-baseline
 * leg of bench.py.  The product library never links, loads or calls it, and it
 * shares no source, header, table or helper with the CUDA path.
 *
 * What it computes (paper section / equation):
 *   - Sec. 2.3, Eq. 9-10: central differences of radius r = order/2 for the
 *     second and first derivative along every axis; ghost nodes pad the grid
 *     by r nodes on every face.
 *   - Sec. 2.1 / Sec. 4 (config_boundary): per face a null Dirichlet, null
 *     Neumann or "none" condition.  Reading used: Dirichlet holds the boundary
 *     node at zero and mirrors odd, p(-j) = -p(j); Neumann mirrors even,
 *     p(-j) = p(j); "none" leaves the ghosts at zero.
 *   - Sec. 2.2, Eq. 5-7: leapfrog update of the damped (variable-density)
 *     wave equation.  Eq. 7 as printed divides only the spatial term by
 *     (1 + eta dt); substituting Eq. 6 into Eq. 5 divides every term, which is
 *     the reading used here:
 *       (1 + eta dt) p[n+1] = kappa (Lap p[n] - grad(ln rho).grad p[n] + f[n])
 *                             + 2 p[n] - (1 - eta dt) p[n-1],
 *     kappa = c^2 dt^2, grad(rho)/rho taken as the FD gradient of ln(rho).
 *     ln(rho) ghosts mirror even on every face.
 *   - Sec. 2.2 (two time levels): p[n+1] overwrites p[n-1] in place.
 *   - Sec. 2.4, Eq. 11-12: point sources add kappa/(1+eta dt) * S(t_n) *
 *     d_k / prod(h) to p[n+1] over their window; receivers record
 *     sum_k d_k p[n+1]_k after the step.  The separable window weights d_k are
 *     built by the Python side (oracle/source.py) and passed in.
 *   - Distributed forcing f(x, t_n) = sum_m F_m(x) T_m(n) (used by the
 *     manufactured-solution tests of Sec. 2.5) enters like the source term.
 *
 * Everything is FP64, plain loops, no blocking or fusion beyond the order above.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { BC_NONE = 0, BC_DIRICHLET = 1, BC_NEUMANN = 2 };

typedef struct {
  int ndim;        /* 2 or 3 */
  int r;           /* stencil radius */
  int64_t n[3];    /* node counts along z, y, x (y = 1 in 2D) */
  int64_t off[3];  /* ghost layers before node 0 along each axis */
  int64_t m[3];    /* padded extents */
  int64_t s[3];    /* strides of the padded array */
  int active[3];   /* axis carries derivatives and ghosts */
} geom;

static int64_t pidx(const geom* g, int64_t z, int64_t y, int64_t x) {
  return (z + g->off[0]) * g->s[0] + (y + g->off[1]) * g->s[1] + (x + g->off[2]);
}

/* Ghost values along every active axis from the face condition (Sec. 2.3). */
static void fill_ghosts(const geom* g, double* f, const int* bc) {
  for (int a = 0; a < 3; ++a) {
    if (!g->active[a]) continue;
    int64_t lo[3] = {0, 0, 0}, hi[3] = {g->n[0], g->n[1], g->n[2]};
    lo[a] = 0;
    hi[a] = 1; /* the loop below runs once along axis a */
    for (int side = 0; side < 2; ++side) {
      int kind = bc[2 * a + side];
      for (int j = 1; j <= g->r; ++j) {
        int64_t ghost = side == 0 ? -j : g->n[a] - 1 + j;
        int64_t mirror = side == 0 ? j : g->n[a] - 1 - j;
        for (int64_t i0 = lo[0]; i0 < hi[0]; ++i0)
          for (int64_t i1 = lo[1]; i1 < hi[1]; ++i1)
            for (int64_t i2 = lo[2]; i2 < hi[2]; ++i2) {
              int64_t q[3] = {i0, i1, i2};
              q[a] = ghost;
              int64_t kg = pidx(g, q[0], q[1], q[2]);
              q[a] = mirror;
              int64_t km = pidx(g, q[0], q[1], q[2]);
              if (kind == BC_DIRICHLET)
                f[kg] = -f[km];
              else if (kind == BC_NEUMANN)
                f[kg] = f[km];
              else
                f[kg] = 0.0;
            }
      }
    }
  }
}

/* Even mirror of a model field into its ghost layers (ln rho). */
static void fill_ghosts_even(const geom* g, double* f) {
  int even[6] = {BC_NEUMANN, BC_NEUMANN, BC_NEUMANN, BC_NEUMANN, BC_NEUMANN, BC_NEUMANN};
  fill_ghosts(g, f, even);
}

/* Zero the boundary nodes of every Dirichlet face. */
static void zero_dirichlet_nodes(const geom* g, double* f, const int* bc) {
  for (int a = 0; a < 3; ++a) {
    if (!g->active[a]) continue;
    for (int side = 0; side < 2; ++side) {
      if (bc[2 * a + side] != BC_DIRICHLET) continue;
      int64_t node = side == 0 ? 0 : g->n[a] - 1;
      int64_t lo[3] = {0, 0, 0}, hi[3] = {g->n[0], g->n[1], g->n[2]};
      lo[a] = node;
      hi[a] = node + 1;
      for (int64_t i0 = lo[0]; i0 < hi[0]; ++i0)
        for (int64_t i1 = lo[1]; i1 < hi[1]; ++i1)
          for (int64_t i2 = lo[2]; i2 < hi[2]; ++i2) f[pidx(g, i0, i1, i2)] = 0.0;
    }
  }
}

/*
 * Window description shared by sources and receivers: for item i and axis a,
 * first[i*3 + a] is the first node of its window and w[(i*3 + a)*len + j] the
 * weight of node first + j (j < len_a; len_y is 1 with weight 1 in 2D).
 */
typedef struct {
  int count;
  const int64_t* first;
  const int* len;    /* per-axis window lengths [3] */
  int len_max;       /* row length of w */
  const double* w;
} windows;

static int window_inside(const geom* g, const windows* wd) {
  for (int i = 0; i < wd->count; ++i)
    for (int a = 0; a < 3; ++a) {
      int64_t f = wd->first[i * 3 + a];
      if (f < 0 || f + wd->len[a] > g->n[a]) return 0;
    }
  return 1;
}

/*
 * Run n_steps leapfrog steps from the given initial levels.
 *
 * Arrays without ghosts ("grid" arrays) are [n0][n1][n2] row-major FP64.
 *   vcoef[0..r]   second-derivative weights v_0..v_r (Eq. 9)
 *   wcoef[1..r]   first-derivative weights w_1..w_r (Eq. 10), wcoef[0] unused;
 *                 may be NULL when lnrho is NULL
 *   bc[6]         face conditions, order z-, z+, y-, y+, x-, x+
 *   eta           damping field (grid), units 1/s
 *   vel           velocity (grid), m/s
 *   lnrho         ln(density) (grid) or NULL for constant density
 *   src/rec       windows (see above); src_sig is [n_src][nt]
 *   force_field   [n_force][grid]; force_sig [n_force][n_steps]
 *   p0, pm1       initial levels p[0], p[-1] (grid) or NULL for zero
 *   seis          [n_steps][n_rec] output; row n holds the receivers after
 *                 step n, i.e. at t_{n+1}
 *   p_last        (grid) output p[n_steps] or NULL; p_prev likewise p[n_steps-1]
 * Returns 0 on success, a positive code on bad arguments.
 */
int oracle_forward(int ndim, const int64_t* shape, const double* spacing, int order,
                   const double* vcoef, const double* wcoef, const int* bc,
                   const double* eta, double dt, const double* vel, const double* lnrho,
                   int n_src, const int64_t* src_first, const int* src_len, int src_len_max,
                   const double* src_w, const double* src_sig, int nt,
                   int n_rec, const int64_t* rec_first, const int* rec_len, int rec_len_max,
                   const double* rec_w,
                   int n_force, const double* force_field, const double* force_sig,
                   const double* p0, const double* pm1,
                   int n_steps, double* seis, double* p_last, double* p_prev,
                   int n_threads) {
  if (ndim != 2 && ndim != 3) return 1;
  if (order < 2 || order % 2 != 0) return 2;
  if (n_steps < 0 || (n_src > 0 && nt < n_steps)) return 3;
  geom g;
  g.ndim = ndim;
  g.r = order / 2;
  double h[3];
  if (ndim == 3) {
    for (int a = 0; a < 3; ++a) {
      g.n[a] = shape[a];
      h[a] = spacing[a];
      g.active[a] = 1;
    }
  } else {
    g.n[0] = shape[0];
    g.n[1] = 1;
    g.n[2] = shape[1];
    h[0] = spacing[0];
    h[1] = 1.0;
    h[2] = spacing[1];
    g.active[0] = 1;
    g.active[1] = 0;
    g.active[2] = 1;
  }
  for (int a = 0; a < 3; ++a) {
    if (g.active[a] && g.n[a] < g.r + 1) return 4;
    g.off[a] = g.active[a] ? g.r : 0;
    g.m[a] = g.n[a] + 2 * g.off[a];
  }
  g.s[2] = 1;
  g.s[1] = g.m[2];
  g.s[0] = g.m[1] * g.m[2];
  windows sw = {n_src, src_first, src_len, src_len_max, src_w};
  windows rw = {n_rec, rec_first, rec_len, rec_len_max, rec_w};
  if (n_src > 0 && !window_inside(&g, &sw)) return 5;
  if (n_rec > 0 && !window_inside(&g, &rw)) return 6;

  const int64_t npad = g.m[0] * g.m[1] * g.m[2];
  const int64_t ngrid = g.n[0] * g.n[1] * g.n[2];
  double* pa = calloc((size_t)npad, sizeof(double)); /* p[n]   */
  double* pb = calloc((size_t)npad, sizeof(double)); /* p[n-1], then p[n+1] */
  double* lr = lnrho ? calloc((size_t)npad, sizeof(double)) : NULL;
  if (!pa || !pb || (lnrho && !lr)) {
    free(pa);
    free(pb);
    free(lr);
    return 7;
  }
  for (int64_t z = 0; z < g.n[0]; ++z)
    for (int64_t y = 0; y < g.n[1]; ++y)
      for (int64_t x = 0; x < g.n[2]; ++x) {
        int64_t k = (z * g.n[1] + y) * g.n[2] + x;
        int64_t kp = pidx(&g, z, y, x);
        if (p0) pa[kp] = p0[k];
        if (pm1) pb[kp] = pm1[k];
        if (lr) lr[kp] = lnrho[k];
      }
  if (lr) fill_ghosts_even(&g, lr);

  double cell = 1.0;
  for (int a = 0; a < 3; ++a)
    if (g.active[a]) cell *= h[a];
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
  const int r = g.r;

  for (int n = 0; n < n_steps; ++n) {
    fill_ghosts(&g, pa, bc);

    /* Eq. 7 (every term divided by 1 + eta dt), in place over p[n-1]. */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t z = 0; z < g.n[0]; ++z)
      for (int64_t y = 0; y < g.n[1]; ++y)
        for (int64_t x = 0; x < g.n[2]; ++x) {
          int64_t k = (z * g.n[1] + y) * g.n[2] + x;
          int64_t kp = pidx(&g, z, y, x);
          double lap = 0.0, adv = 0.0;
          for (int a = 0; a < 3; ++a) {
            if (!g.active[a]) continue;
            int64_t st = g.s[a];
            double d2 = vcoef[0] * pa[kp];
            for (int j = 1; j <= r; ++j) d2 += vcoef[j] * (pa[kp + j * st] + pa[kp - j * st]);
            lap += d2 / (h[a] * h[a]);
            if (lr) {
              double dp = 0.0, dl = 0.0;
              for (int j = 1; j <= r; ++j) {
                dp += wcoef[j] * (pa[kp + j * st] - pa[kp - j * st]);
                dl += wcoef[j] * (lr[kp + j * st] - lr[kp - j * st]);
              }
              adv += (dl / (2.0 * h[a])) * (dp / (2.0 * h[a]));
            }
          }
          double kap = vel[k] * vel[k] * dt * dt;
          double e = eta[k] * dt;
          pb[kp] = (kap * (lap - adv) + 2.0 * pa[kp] - (1.0 - e) * pb[kp]) / (1.0 + e);
        }

    /* Eq. 11: point sources, S(t_n) into p[n+1]. */
    for (int i = 0; i < n_src; ++i) {
      double sig = src_sig[(int64_t)i * nt + n];
      const int64_t* f = src_first + i * 3;
      const double* wz = src_w + ((int64_t)i * 3 + 0) * src_len_max;
      const double* wy = src_w + ((int64_t)i * 3 + 1) * src_len_max;
      const double* wx = src_w + ((int64_t)i * 3 + 2) * src_len_max;
      for (int a = 0; a < src_len[0]; ++a)
        for (int b = 0; b < src_len[1]; ++b)
          for (int c = 0; c < src_len[2]; ++c) {
            int64_t z = f[0] + a, y = f[1] + b, x = f[2] + c;
            int64_t k = (z * g.n[1] + y) * g.n[2] + x;
            double kap = vel[k] * vel[k] * dt * dt;
            double e = eta[k] * dt;
            pb[pidx(&g, z, y, x)] += kap / (1.0 + e) * sig * (wz[a] * wy[b] * wx[c]) / cell;
          }
    }
    /* Distributed forcing sum_m F_m(x) T_m(t_n), same scaling as a source. */
    for (int mth = 0; mth < n_force; ++mth) {
      double tm = force_sig[(int64_t)mth * n_steps + n];
      const double* fm = force_field + (int64_t)mth * ngrid;
      for (int64_t z = 0; z < g.n[0]; ++z)
        for (int64_t y = 0; y < g.n[1]; ++y)
          for (int64_t x = 0; x < g.n[2]; ++x) {
            int64_t k = (z * g.n[1] + y) * g.n[2] + x;
            double kap = vel[k] * vel[k] * dt * dt;
            double e = eta[k] * dt;
            pb[pidx(&g, z, y, x)] += kap / (1.0 + e) * fm[k] * tm;
          }
    }
    zero_dirichlet_nodes(&g, pb, bc);

    /* Two time levels: the new level now lives in pb. */
    double* t = pa;
    pa = pb;
    pb = t;

    /* Eq. 12: receivers sample p[n+1]. */
    for (int i = 0; i < n_rec; ++i) {
      const int64_t* f = rec_first + i * 3;
      const double* wz = rec_w + ((int64_t)i * 3 + 0) * rec_len_max;
      const double* wy = rec_w + ((int64_t)i * 3 + 1) * rec_len_max;
      const double* wx = rec_w + ((int64_t)i * 3 + 2) * rec_len_max;
      double acc = 0.0;
      for (int a = 0; a < rec_len[0]; ++a)
        for (int b = 0; b < rec_len[1]; ++b)
          for (int c = 0; c < rec_len[2]; ++c)
            acc += wz[a] * wy[b] * wx[c] * pa[pidx(&g, f[0] + a, f[1] + b, f[2] + c)];
      seis[(int64_t)n * n_rec + i] = acc;
    }
  }

  for (int64_t z = 0; z < g.n[0]; ++z)
    for (int64_t y = 0; y < g.n[1]; ++y)
      for (int64_t x = 0; x < g.n[2]; ++x) {
        int64_t k = (z * g.n[1] + y) * g.n[2] + x;
        int64_t kp = pidx(&g, z, y, x);
        if (p_last) p_last[k] = pa[kp];
        if (p_prev) p_prev[k] = pb[kp];
      }
  free(pa);
  free(pb);
  free(lr);
  return 0;
}
