/*
 * CPU oracle, one dimension. TEST INFRASTRUCTURE ONLY (see ch_oracle.h).
 *
 * Every routine is the paper's definition written out in FP64 with no blocking,
 * fusion or reordering: the matrices of Section 2.1 / Eq. 3.2 are assembled in band
 * form and each implicit step is solved by Gaussian elimination with partial pivoting.
 */
#include "ch_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

/* ---------------------------------------------------------------- D_h (Eq. 3.2) */

int orc1d_dh_apply(int n, const double* u, double* out) {
  if (n < 1 || !u || !out) return 1;
  const double h = 1.0 / (n + 1);
  const double ih2 = 1.0 / (h * h);
  for (int j = 0; j < n; ++j) {
    const double left = (j > 0) ? u[j - 1] : 0.0;       /* boundary value u = 0 */
    const double right = (j < n - 1) ? u[j + 1] : 0.0;
    out[j] = ih2 * (left - 2.0 * u[j] + right);
  }
  return 0;
}

/* ------------------------------------------- banded Gaussian elimination (pivoting) */

int orc_band_solve(int n, int kl, int ku, double* a, double* b) {
  if (n < 1 || kl < 0 || ku < 0 || !a || !b) return 1;
  const int w = 2 * kl + ku + 1;
#define A(i, j) a[(size_t)(i) * w + ((j) - (i) + kl)]
  for (int k = 0; k < n; ++k) {
    const int last_row = (k + kl < n - 1) ? k + kl : n - 1;
    const int last_col = (k + kl + ku < n - 1) ? k + kl + ku : n - 1;
    int piv = k;
    double best = fabs(A(k, k));
    for (int i = k + 1; i <= last_row; ++i) {
      if (fabs(A(i, k)) > best) { best = fabs(A(i, k)); piv = i; }
    }
    if (best == 0.0) return 2;
    if (piv != k) {
      for (int j = k; j <= last_col; ++j) { double t = A(k, j); A(k, j) = A(piv, j); A(piv, j) = t; }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int i = k + 1; i <= last_row; ++i) {
      const double l = A(i, k) / A(k, k);
      if (l == 0.0) continue;
      A(i, k) = 0.0;
      for (int j = k + 1; j <= last_col; ++j) A(i, j) -= l * A(k, j);
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    const int last_col = (i + kl + ku < n - 1) ? i + kl + ku : n - 1;
    double s = b[i];
    for (int j = i + 1; j <= last_col; ++j) s -= A(i, j) * b[j];
    b[i] = s / A(i, i);
  }
#undef A
  return 0;
}

/* ------------------------------------------------------------- matrix assembly */

/* Band rows (kl = ku = 2) of  I + c2 D_h^2 - c1 D_h diag(w)  where w may be NULL (w = 1).
 * D_h^2 rows: h^-4 [1 -4 6 -4 1], first/last rows h^-4 [5 -4 1] (zero boundary values).
 * (D_h diag(w))_{j,l} = h^-2 { w_{j-1}, -2 w_j, w_{j+1} } at l = j-1, j, j+1. */
static void assemble(int n, double c1, double c2, const double* w, double* a) {
  const int kl = 2, ku = 2, wdt = 2 * kl + ku + 1;
  const double h = 1.0 / (n + 1);
  const double ih2 = 1.0 / (h * h);
  const double ih4 = ih2 * ih2;
  memset(a, 0, sizeof(double) * (size_t)n * wdt);
#define A(i, j) a[(size_t)(i) * wdt + ((j) - (i) + kl)]
  for (int j = 0; j < n; ++j) {
    /* D_h^2 = D_h D_h, entry (j,l) = sum_m D(j,m) D(m,l) over interior m */
    for (int l = j - 2; l <= j + 2; ++l) {
      if (l < 0 || l >= n) continue;
      double d2 = 0.0;
      for (int m = j - 1; m <= j + 1; ++m) {
        if (m < 0 || m >= n) continue;
        const double djm = (m == j) ? -2.0 : 1.0;
        const int dml = m - l;
        const double dm = (dml == 0) ? -2.0 : ((dml == 1 || dml == -1) ? 1.0 : 0.0);
        d2 += djm * dm;
      }
      A(j, l) += c2 * ih4 * d2;
    }
    A(j, j) += 1.0;
    for (int l = j - 1; l <= j + 1; ++l) {
      if (l < 0 || l >= n) continue;
      const double dl = (l == j) ? -2.0 : 1.0;
      const double wl = w ? w[l] : 1.0;
      A(j, l) -= c1 * ih2 * dl * wl;
    }
  }
#undef A
}

static void add_forcing(int n, double dt, double t, const orc_forcing* f, double* rhs) {
  if (!f || f->nmodes <= 0) return;
  const double h = 1.0 / (n + 1);
  for (int j = 0; j < n; ++j) {
    const double x = (j + 1) * h;
    double g = 0.0;
    for (int i = 0; i < f->nmodes; ++i) g += f->a[i] * exp(f->b[i] * t) * sin(f->m[i] * PI * x);
    rhs[j] += dt * g;
  }
}

/* ----------------------------------------------------------------- time steps */

/* The linear step M Y = b of Eq. 2.4 / 2.5, M = I + e2dt D_h^2 - cdt D_h diag(w) (w = 1 when
 * NULL; `a` holds M in band form), taken from its residual instead of one elimination: Y_0 = u^n,
 * Y_{m+1} = Y_m - M^{-1} H(Y_m) with H(Y) = Y + e2dt D_h (D_h Y) - cdt D_h (w Y) - b, stopped by
 * the Newton rule of the nonlinear step. The same step with other rounding: the FP64 residual
 * fixes the attainable accuracy, as in a solver that refines a low-precision solve. */
static int linear_by_residual(const orc_params* p, int n, double e2dt, double cdt, const double* w,
                              const double* a, const double* b, const double* u, double* out,
                              orc_stats* st) {
  const int wdt = 7;
  double* lu = (double*)malloc(sizeof(double) * (size_t)n * wdt);
  double* y = (double*)malloc(sizeof(double) * n);
  double* hh = (double*)malloc(sizeof(double) * n);
  double* dy = (double*)malloc(sizeof(double) * n);
  double* d2y = (double*)malloc(sizeof(double) * n);
  double* wy = (double*)malloc(sizeof(double) * n);
  double* dwy = (double*)malloc(sizeof(double) * n);
  int rc = 0, m = 0, ok = 0;
  double prev = 0.0;
  if (!lu || !y || !hh || !dy || !d2y || !wy || !dwy) { rc = 1; goto done; }
  memcpy(y, u, sizeof(double) * n);
  while (m < p->newton_max) {
    orc1d_dh_apply(n, y, dy);
    orc1d_dh_apply(n, dy, d2y);
    for (int j = 0; j < n; ++j) wy[j] = (w ? w[j] : 1.0) * y[j];
    orc1d_dh_apply(n, wy, dwy);
    for (int j = 0; j < n; ++j) hh[j] = y[j] + e2dt * d2y[j] - cdt * dwy[j] - b[j];
    memcpy(lu, a, sizeof(double) * (size_t)n * wdt); /* orc_band_solve factors in place */
    rc = orc_band_solve(n, 2, 2, lu, hh);
    if (rc) break;
    double diff = 0.0;
    for (int j = 0; j < n; ++j) {
      y[j] -= hh[j];
      if (fabs(hh[j]) > diff) diff = fabs(hh[j]);
    }
    ++m;
    if (diff <= p->newton_tol) { ok = 1; break; }
    if (m >= 2 && diff <= sqrt(p->newton_tol) && diff > 0.5 * prev) { ok = 1; break; }
    prev = diff;
  }
  if (st) {
    st->newton_total += m;
    if (m > st->newton_max_seen) st->newton_max_seen = m;
  }
  if (!rc && !ok) rc = 3;
  if (!rc) memcpy(out, y, sizeof(double) * n);
done:
  free(lu); free(y); free(hh); free(dy); free(d2y); free(wy); free(dwy);
  return rc;
}

int orc1d_step(const orc_params* p, int scheme, double dt, double t_next, const double* u,
               double* out, const orc_forcing* f, orc_stats* st) {
  if (!p || !u || !out || p->n < 1 || dt <= 0.0) return 1;
  const int n = p->n;
  const double e2 = p->eps * p->eps;
  const int wdt = 7;
  double* a = (double*)malloc(sizeof(double) * (size_t)n * wdt);
  double* rhs = (double*)malloc(sizeof(double) * n);
  double* tmp = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double* y = (double*)malloc(sizeof(double) * n);
  int rc = 0;
  if (!a || !rhs || !tmp || !w || !y) { rc = 1; goto done; }

  if (scheme == ORC_LIN1) {
    /* Eq. 2.4 */
    orc1d_dh_apply(n, u, tmp);
    for (int j = 0; j < n; ++j) { rhs[j] = u[j] - dt * tmp[j]; w[j] = u[j] * u[j]; }
    add_forcing(n, dt, t_next, f, rhs);
    assemble(n, dt, e2 * dt, p->frozen ? NULL : w, a);
    if (p->newton_form == 1) {
      rc = linear_by_residual(p, n, e2 * dt, dt, p->frozen ? NULL : w, a, rhs, u, out, st);
    } else {
      rc = orc_band_solve(n, 2, 2, a, rhs);
      if (!rc) memcpy(out, rhs, sizeof(double) * n);
    }
  } else if (scheme == ORC_LIN2) {
    /* Eq. 2.5 (D_h on the implicit 2 dt term) */
    for (int j = 0; j < n; ++j) w[j] = p->frozen ? u[j] : u[j] * u[j] * u[j];
    orc1d_dh_apply(n, w, tmp);
    orc1d_dh_apply(n, u, y);
    for (int j = 0; j < n; ++j) rhs[j] = u[j] + dt * tmp[j] - 3.0 * dt * y[j];
    add_forcing(n, dt, t_next, f, rhs);
    assemble(n, 2.0 * dt, e2 * dt, NULL, a);
    if (p->newton_form == 1) {
      rc = linear_by_residual(p, n, e2 * dt, 2.0 * dt, NULL, a, rhs, u, out, st);
    } else {
      rc = orc_band_solve(n, 2, 2, a, rhs);
      if (!rc) memcpy(out, rhs, sizeof(double) * n);
    }
  } else if (scheme == ORC_NL) {
    /* Eq. 3.17: Yhat = (I - dt D_h) u^n; Newton of Eq. 3.18 from Y_0 = u^n. */
    double* yhat = (double*)malloc(sizeof(double) * n);
    if (!yhat) { rc = 1; goto done; }
    orc1d_dh_apply(n, u, tmp);
    for (int j = 0; j < n; ++j) yhat[j] = u[j] - dt * tmp[j];
    add_forcing(n, dt, t_next, f, yhat);
    memcpy(y, u, sizeof(double) * n);
    int m = 0, ok = 0;
    double prev = 0.0;
    while (m < p->newton_max) {
      /* Y_{m+1} = (I + eps^2 dt D_h^2 - 3 dt D_h diag(Y_m^2))^{-1} (Yhat - 2 dt D_h diag(Y_m^2) Y_m) */
      for (int j = 0; j < n; ++j) {
        w[j] = p->frozen ? 1.0 : y[j] * y[j];
        tmp[j] = w[j] * y[j];
      }
      orc1d_dh_apply(n, tmp, rhs);
      double* nxt = tmp;
      for (int j = 0; j < n; ++j) nxt[j] = yhat[j] - 2.0 * dt * rhs[j];
      if (p->frozen) {
        /* frozen model: Y^3 -> Y, so H is linear and Newton solves (I + e2 dt D^2 - dt D) Y = Yhat */
        memcpy(nxt, yhat, sizeof(double) * n);
        assemble(n, dt, e2 * dt, NULL, a);
      } else {
        assemble(n, 3.0 * dt, e2 * dt, w, a);
      }
      if (p->newton_form == 1 && !p->frozen) {
        /* H(Y) = Y + eps^2 dt D_h (D_h Y) - dt D_h Y^3 - Yhat (Eq. 3.17); Y_{m+1} = Y_m - J^{-1} H */
        double* dy = (double*)malloc(sizeof(double) * n);
        double* d2y = (double*)malloc(sizeof(double) * n);
        double* y3 = (double*)malloc(sizeof(double) * n);
        double* dy3 = (double*)malloc(sizeof(double) * n);
        if (!dy || !d2y || !y3 || !dy3) { free(dy); free(d2y); free(y3); free(dy3); rc = 1; break; }
        orc1d_dh_apply(n, y, dy);
        orc1d_dh_apply(n, dy, d2y);
        for (int j = 0; j < n; ++j) y3[j] = y[j] * y[j] * y[j];
        orc1d_dh_apply(n, y3, dy3);
        for (int j = 0; j < n; ++j) nxt[j] = y[j] + e2 * dt * d2y[j] - dt * dy3[j] - yhat[j];
        rc = orc_band_solve(n, 2, 2, a, nxt);
        for (int j = 0; j < n; ++j) nxt[j] = y[j] - nxt[j];
        free(dy); free(d2y); free(y3); free(dy3);
      } else {
        rc = orc_band_solve(n, 2, 2, a, nxt);
      }
      if (rc) break;
      double diff = 0.0;
      for (int j = 0; j < n; ++j) {
        const double d = fabs(nxt[j] - y[j]);
        if (d > diff) diff = d;
      }
      memcpy(y, nxt, sizeof(double) * n);
      ++m;
      if (diff <= p->newton_tol) { ok = 1; break; }
      /* Rounding floor: once below sqrt(tol), an increment that does not halve the previous
       * one is rounding noise of the FP64 residual; the iterate is converged. */
      if (m >= 2 && diff <= sqrt(p->newton_tol) && diff > 0.5 * prev) { ok = 1; break; }
      prev = diff;
    }
    free(yhat);
    if (st) {
      st->newton_total += m;
      if (m > st->newton_max_seen) st->newton_max_seen = m;
    }
    if (!rc && !ok) rc = 3;
    if (!rc) memcpy(out, y, sizeof(double) * n);
  } else {
    rc = 1;
  }
  if (st && !rc) st->steps += 1;
done:
  free(a); free(rhs); free(tmp); free(w); free(y);
  return rc;
}

int orc1d_propagate(const orc_params* p, int scheme, double dt, int nsteps, double t0,
                    const double* u_in, double* u_out, const orc_forcing* f, orc_stats* st) {
  if (!p || nsteps < 0 || !u_in || !u_out) return 1;
  const int n = p->n;
  double* cur = (double*)malloc(sizeof(double) * n);
  double* nxt = (double*)malloc(sizeof(double) * n);
  if (!cur || !nxt) { free(cur); free(nxt); return 1; }
  memcpy(cur, u_in, sizeof(double) * n);
  int rc = 0;
  for (int s = 0; s < nsteps && !rc; ++s) {
    rc = orc1d_step(p, scheme, dt, t0 + (s + 1) * dt, cur, nxt, f, st);
    double* t = cur; cur = nxt; nxt = t;
  }
  if (!rc) memcpy(u_out, cur, sizeof(double) * n);
  free(cur); free(nxt);
  return rc;
}

/* ------------------------------------------------------------- Parareal (Eq. 2.2) */

static int fine(const orc_params* p, double t0, const double* u, double* out, orc_stats* st) {
  const double dT = p->T / p->N;
  return orc1d_propagate(p, p->fine_scheme, dT / p->J, p->J, t0, u, out, NULL, st);
}

static int coarse(const orc_params* p, double t0, const double* u, double* out) {
  const double dT = p->T / p->N;
  return orc1d_propagate(p, p->coarse_scheme, dT / p->coarse_steps, p->coarse_steps, t0, u, out,
                         NULL, NULL);
}

int orc1d_fine_solution(const orc_params* p, const double* u0, double* Uf, orc_stats* st) {
  if (!p || !u0 || !Uf || p->N < 1 || p->J < 1) return 1;
  const int n = p->n;
  memcpy(Uf, u0, sizeof(double) * n);
  for (int s = 0; s < p->N; ++s) {
    int rc = fine(p, s * p->T / p->N, Uf + (size_t)s * n, Uf + (size_t)(s + 1) * n, st);
    if (rc) return rc;
  }
  return 0;
}

static void errors(const orc_params* p, const double* U, const double* Uf, double* l2, double* mx) {
  const int n = p->n;
  const double h = 1.0 / (n + 1);
  double el2 = 0.0, emx = 0.0;
  for (int s = 0; s <= p->N; ++s) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) {
      const double e = U[(size_t)s * n + j] - Uf[(size_t)s * n + j];
      acc += e * e;
      if (fabs(e) > emx) emx = fabs(e);
    }
    const double v = sqrt(h * acc);
    if (v > el2) el2 = v;
  }
  *l2 = el2;
  *mx = emx;
}

int orc1d_parareal(const orc_params* p, const double* u0, const double* Uf, double* U,
                   orc_result* res) {
  if (!p || !u0 || !U || !res || p->N < 1 || p->J < 1 || p->coarse_steps < 1) return 1;
  if (p->max_iters < 0 || p->max_iters > p->N || p->N > 1023) return 1;
  const int n = p->n, N = p->N;
  const size_t sz = (size_t)(N + 1) * n;
  memset(res, 0, sizeof(*res));
  double* Gold = (double*)malloc(sizeof(double) * (size_t)N * n);  /* G(U_n^k) */
  double* Fk = (double*)malloc(sizeof(double) * (size_t)N * n);    /* F(U_n^k) */
  double* Unew = (double*)malloc(sizeof(double) * sz);
  double* g = (double*)malloc(sizeof(double) * n);
  int rc = 0;
  if (!Gold || !Fk || !Unew || !g) { rc = 1; goto out; }

  /* U^0: coarse sweep from u^0 (Section 4) */
  memcpy(U, u0, sizeof(double) * n);
  for (int s = 0; s < N && !rc; ++s) {
    rc = coarse(p, s * p->T / N, U + (size_t)s * n, U + (size_t)(s + 1) * n);
    if (!rc) memcpy(Gold + (size_t)s * n, U + (size_t)(s + 1) * n, sizeof(double) * n);
  }
  if (rc) goto out;
  if (Uf) errors(p, U, Uf, &res->err_l2[0], &res->err_max[0]);

  for (int k = 0; k < p->max_iters; ++k) {
    /* fine propagation of the current iterate on the slices not yet exact (n >= k) */
    for (int s = k; s < N && !rc; ++s)
      rc = fine(p, s * p->T / N, U + (size_t)s * n, Fk + (size_t)s * n, &res->st);
    if (rc) goto out;
    /* sequential correction: U_{s+1}^{k+1} = G(U_s^{k+1}) + F(U_s^k) - G(U_s^k), evaluated as
     * F + (G_new - G_old) so that an exact coarse cancellation leaves F unchanged. */
    memcpy(Unew, U, sizeof(double) * (size_t)(k + 1) * n);
    for (int s = k; s < N && !rc; ++s) {
      rc = coarse(p, s * p->T / N, Unew + (size_t)s * n, g);
      if (rc) break;
      double* dst = Unew + (size_t)(s + 1) * n;
      for (int j = 0; j < n; ++j)
        dst[j] = Fk[(size_t)s * n + j] + (g[j] - Gold[(size_t)s * n + j]);
      memcpy(Gold + (size_t)s * n, g, sizeof(double) * n);
    }
    if (rc) goto out;
    double inc = 0.0;
    for (size_t i = 0; i < sz; ++i) {
      const double d = fabs(Unew[i] - U[i]);
      if (d > inc) inc = d;
    }
    memcpy(U, Unew, sizeof(double) * sz);
    res->iterations = k + 1;
    res->inc[k] = inc;
    if (Uf) errors(p, U, Uf, &res->err_l2[k + 1], &res->err_max[k + 1]);
    if (p->tol > 0.0 && inc < p->tol) { res->converged = 1; break; }
  }
out:
  free(Gold); free(Fk); free(Unew); free(g);
  return rc;
}

/* ---------------------------------------------------------------------- energy */

double orc1d_energy(int n, double eps, const double* u) {
  const double h = 1.0 / (n + 1);
  double bulk = 0.0, grad = 0.0;
  for (int j = 0; j < n; ++j) {
    const double q = u[j] * u[j] - 1.0;
    bulk += 0.25 * q * q;
  }
  for (int j = 0; j <= n; ++j) {  /* u^T (-D_h) u = h^-2 sum (u_{j+1} - u_j)^2, zero boundary */
    const double a = (j > 0) ? u[j - 1] : 0.0;
    const double b = (j < n) ? u[j] : 0.0;
    grad += (b - a) * (b - a);
  }
  return h * bulk + 0.5 * eps * eps * grad / h;
}
