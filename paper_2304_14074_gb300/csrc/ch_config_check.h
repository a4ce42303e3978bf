// Argument checks of ch_config shared by every entry point that takes one (ch_parareal.h).
#pragma once
#include <cmath>
#include <string>

#include "ch_parareal.h"

namespace chcfg {

inline bool finite_pos(double x) { return x > 0.0 && std::isfinite(x); }

// Fields every call uses: grid, eps, the Newton controls, precision and the 2D inner solve.
inline bool valid_common(const ch_config* c, bool (*supported_2d)(int), std::string& why) {
  if (!c) { why = "cfg is NULL"; return false; }
  if (c->dim != 1 && c->dim != 2) { why = "dim must be 1 or 2"; return false; }
  if (c->dim == 1 && (c->n < 1 || c->n > 2048)) { why = "n must be in 1..2048"; return false; }
  if (c->dim == 2 && !supported_2d(c->n)) { why = "2D needs n + 1 in {16, 32, ..., 512}"; return false; }
  if (!finite_pos(c->eps)) { why = "eps must be finite and > 0"; return false; }
  if (c->newton_max < 1 || c->newton_max > 1000) { why = "newton_max must be in 1..1000"; return false; }
  if (!finite_pos(c->newton_tol)) { why = "newton_tol must be finite and > 0"; return false; }
  if (c->precision != 0 && c->precision != 1) { why = "precision must be 0 or 1"; return false; }
  if (!std::isfinite(c->lin_tol) || c->lin_tol >= 1.0) { why = "lin_tol must be finite and < 1"; return false; }
  if (c->lin_max > 10000) { why = "lin_max must be <= 10000"; return false; }
  return true;
}

// Fields of a Parareal run: time interval, slices, steps, variant, stop rules.
inline bool valid_run(const ch_config* c, bool (*supported_2d)(int), std::string& why) {
  if (!valid_common(c, supported_2d, why)) return false;
  if (!finite_pos(c->T)) { why = "T must be finite and > 0"; return false; }
  if (c->n_slices < 1 || c->n_slices > CH_MAX_ITERS - 1) { why = "n_slices must be in 1..1023"; return false; }
  if (c->fine_steps < 1 || c->coarse_steps < 1) { why = "fine_steps and coarse_steps must be >= 1"; return false; }
  if (c->variant < CH_PA_I || c->variant > CH_NPA_II) { why = "unknown variant"; return false; }
  if (c->max_iters < 1 || c->max_iters > c->n_slices) { why = "max_iters must be in 1..n_slices"; return false; }
  if (!std::isfinite(c->tol) || !std::isfinite(c->err_tol)) { why = "tol and err_tol must be finite"; return false; }
  return true;
}

// Inner CG controls of the 2D solver (defaults for values <= 0).
inline double lin_tol_of(const ch_config* c) { return c->lin_tol > 0.0 ? c->lin_tol : 1e-3; }
inline int lin_max_of(const ch_config* c) { return c->lin_max > 0 ? c->lin_max : 60; }

}  // namespace chcfg
