// C ABI of the Parareal library (declared in include/ch_parareal.h): handle lifetime, device
// memory, the iteration driver (CUDA graphs replayed per Parareal iteration) and statistics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ch1d.cuh"
#include "ch2d.cuh"
#include "ch_parareal.h"
#include "ch_trace.cuh"
#include "ch_config_check.h"
#include "gtheta.cuh"

using chg::Ctrl;
using chg::Params1D;
using chg::ProblemState;

struct ch_parareal {
  ch_config cfg{};
  int B = 0;
  cudaStream_t st = nullptr;
  int device = 0;
  Params1D p{};
  size_t pts = 0;
  double* U = nullptr;     // [B][N+1][pts]
  double* F = nullptr;     // [B][N][pts]
  double* Gold = nullptr;  // [B][N][pts]
  double* Uref = nullptr;  // [B][N+1][pts]
  Ctrl* ctrl = nullptr;
  ProblemState ps{};
  void* ps_block = nullptr;
  int* host_active = nullptr;  // mapped pinned
  int* host_active_dev = nullptr;
  std::vector<int> initial_set;
  bool ref_valid = false;
  bool ran = false;
  int grid = 0;
  size_t ps_bytes = 0;
  bool tuned = false;  // 1D fine-sweep launch configuration chosen by measurement
  // Each iteration replays two graphs, [fine sweep] then [coarse sweep + correction, tally];
  // timing events are recorded on the stream between them (events inside a graph cannot time).
  cudaGraphExec_t gfine = nullptr;
  cudaGraphExec_t gcoarse = nullptr;
  int graph_ref = -1;  // whether the captured coarse graph reads the reference solution
  std::vector<cudaEvent_t> ev;  // ev[0] = start, ev[k+1] = end of iteration k (k = 0: coarse sweep)
  cudaEvent_t ph[3] = {nullptr, nullptr, nullptr};  // before fine, after fine, after coarse
  double fine_ms = 0.0, coarse_ms = 0.0;
  int kernel_launches = 0;
  std::vector<int> active_before;  // active problems entering each iteration
  int iters_done = 0;
  ch_status sticky = CH_OK;
  std::string msg;
  // two-dimensional path
  int dim = 1;
  chg2::Prop2D* p2 = nullptr;
  double* W = nullptr;          // [B N][pts] gathered states being propagated
  double* acc = nullptr;        // [B][3] running {inc, err_l2, err_max} of an iteration
  double* cpart = nullptr;      // correction partials
  int* dlist = nullptr;         // [B] problem list
  long long* doff = nullptr;    // [B N] element offsets for gather / scatter
  std::vector<std::vector<double>> h_inc, h_el2, h_emx;
  std::vector<int> h_iters, h_conv;
  unsigned long long fine_newton = 0;  // Newton iterations (summed over units) of the fine sweeps
  long long fine_cg = 0;               // CG iterations (summed over units) of the fine sweeps
  // learned coarse propagator (2D): null = plain coarse step
  chg3::GTheta* gt = nullptr;
  int gt_form = CH_GTHETA_RESIDUAL;
  double* Wtmp = nullptr;  // [B][pts] G_theta inputs of the correction form
  std::vector<int> h_learned, h_fallback;
  long long gt_launches = 0;
  long long aux_launches = 0;  // gather / scatter / correction kernels of the 2D driver
  std::vector<double> eps_prob;   // per-problem eps (2D, ch_parareal_set_eps); empty = cfg.eps
  double* eps2u_dev = nullptr;    // eps^2 of the gathered work rows [B N]
};

namespace {

ch_status fail(ch_parareal* h, ch_status s, const std::string& m) {
  if (h && h->sticky == CH_OK) {
    h->sticky = s;
    h->msg = m;
  }
  return s;
}

// A Newton or linear-solve failure is a property of the data that was propagated, not of the
// handle: new initial states clear it. Every other error stays.
void clear_data_error(ch_parareal* h) {
  if (h->sticky == CH_ERR_NEWTON || h->sticky == CH_ERR_LINSOLVE) {
    h->sticky = CH_OK;
    h->msg.clear();
  }
}

ch_status cuda_fail(ch_parareal* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) return fail(h, CH_ERR_OOM, m);
  return fail(h, CH_ERR_CUDA, m);
}

#define CH_CUDA(h, call)                                  \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

int fine_of(int v) { return (v == CH_PA_I) ? chg::SCHEME_LIN1 : (v == CH_NPA_I || v == CH_NPA_II) ? chg::SCHEME_NL : chg::SCHEME_LIN2; }
int coarse_of(int v) { return (v == CH_PA_II) ? chg::SCHEME_LIN2 : (v == CH_NPA_II) ? chg::SCHEME_NL : chg::SCHEME_LIN1; }

bool valid_common(const ch_config* c, std::string& why) { return chcfg::valid_common(c, chg2::supported_n, why); }

Params1D make_params(const ch_config* c, int B) {
  Params1D p{};
  p.n = c->n;
  p.B = B;
  p.N = c->n_slices;
  p.J = c->fine_steps;
  p.coarse_steps = c->coarse_steps;
  p.fine_scheme = fine_of(c->variant);
  p.coarse_scheme = coarse_of(c->variant);
  p.precision = c->precision;
  p.frozen = c->frozen ? 1 : 0;
  p.newton_max = c->newton_max;
  p.maxit = c->max_iters;
  p.eps2 = c->eps * c->eps;
  p.h = 1.0 / (c->n + 1);
  const double dT = (c->n_slices > 0) ? c->T / c->n_slices : 0.0;
  p.dt = (c->fine_steps > 0) ? dT / c->fine_steps : 0.0;
  p.dtc = (c->coarse_steps > 0) ? dT / c->coarse_steps : 0.0;
  p.newton_tol = c->newton_tol;
  p.tol = c->tol;
  p.err_tol = c->err_tol;
  return p;
}

chg2::Params2D params2d(const ch_config* c) {
  chg2::Params2D q{};
  q.n = c->n;
  q.frozen = c->frozen ? 1 : 0;
  q.newton_max = c->newton_max;
  // Inexact Newton: each CG solve reduces the preconditioned residual by lin_tol (default 1e-3);
  // the Newton error then contracts by about that factor per iteration down to the FP64
  // residual floor.
  q.cg_max = chcfg::lin_max_of(c);
  q.eps2 = c->eps * c->eps;
  q.h = 1.0 / (c->n + 1);
  q.newton_tol = c->newton_tol;
  q.cg_tol = chcfg::lin_tol_of(c);
  return q;
}

ch_status device_status(ch_parareal* h, unsigned status) {
  if (status & chg2::ST_TIMEOUT) return fail(h, CH_ERR_TIMEOUT, "a grid barrier of the 2D solver timed out");
  if (status & chg::ST_NONFINITE) return fail(h, CH_ERR_LINSOLVE, "a solve produced a non-finite value");
  if (status & chg::ST_NEWTON) return fail(h, CH_ERR_NEWTON, "a Newton solve reached newton_max");
  return CH_OK;
}

// ------------------------------------------------------------------ two-dimensional driver

int fine2(const ch_parareal* h) { return fine_of(h->cfg.variant); }
int coarse2(const ch_parareal* h) { return coarse_of(h->cfg.variant); }

// Work rows W[i] = U[b][s] for (b, s) in `units`, via element offsets.
ch_status gather_units(ch_parareal* h, double* src, const std::vector<long long>& off, bool to_w) {
  if (off.empty()) return CH_OK;
  CH_CUDA(h, cudaMemcpyAsync(h->doff, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, h->st));
  h->aux_launches += 1;
  if (to_w && h->eps2u_dev) {
    // eps^2 of each work row, from the problem its offset (into U) belongs to
    const size_t us = (size_t)(h->p.N + 1) * h->pts;
    std::vector<double> e2(off.size());
    for (size_t i = 0; i < off.size(); ++i) {
      const double e = h->eps_prob[(size_t)off[i] / us];
      e2[i] = e * e;
    }
    CH_CUDA(h, cudaMemcpyAsync(h->eps2u_dev, e2.data(), e2.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
  }
  if (to_w) {
    CH_CUDA(h, chg2::launch_gather(h->W, src, h->doff, (int)off.size(), h->pts, h->st));
  } else {
    CH_CUDA(h, chg2::launch_scatter(src, h->W, h->doff, (int)off.size(), h->pts, h->st));
  }
  return CH_OK;
}

ch_status prop2(ch_parareal* h, int units, int scheme, double dt, int nsteps, size_t row0 = 0) {
  CH_CUDA(h, h->p2->propagate(h->W + row0 * h->pts, units, scheme, dt, nsteps, h->st));
  return CH_OK;
}

// One coarse step of the work rows W[0, nb): rows [0, nl) with G_theta, the rest with the plain
// coarse scheme. The correction form runs the plain step on every row and adds R of the row's
// input to the first nl.
ch_status coarse_rows(ch_parareal* h, int nb, int nl) {
  const int scheme = coarse_of(h->cfg.variant);
  if (nl > 0 && h->gt_form == CH_GTHETA_CORRECTION) {
    CH_CUDA(h, cudaMemcpyAsync(h->Wtmp, h->W, (size_t)nl * h->pts * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    ch_status s = prop2(h, nb, scheme, h->p.dtc, h->p.coarse_steps);
    if (s != CH_OK) return s;
    CH_CUDA(h, h->gt->forward64(h->Wtmp, h->W, h->W, nl, h->cfg.n, h->st));
    h->gt_launches += chg3::GTheta::kForwardKernels;
    return CH_OK;
  }
  if (nl > 0) {
    CH_CUDA(h, h->gt->forward64(h->W, nullptr, h->W, nl, h->cfg.n, h->st));
    h->gt_launches += chg3::GTheta::kForwardKernels;
  }
  if (nb > nl) return prop2(h, nb - nl, scheme, h->p.dtc, h->p.coarse_steps, (size_t)nl);
  return CH_OK;
}

ch_status reference2d(ch_parareal* h) {
  const int B = h->B, N = h->p.N;
  const size_t pts = h->pts, us = (size_t)(N + 1) * pts;
  std::vector<long long> off(B);
  for (int b = 0; b < B; ++b) off[b] = (long long)(b * us);
  CH_CUDA(h, cudaMemcpy2DAsync(h->Uref, us * sizeof(double), h->U, us * sizeof(double), pts * sizeof(double), B,
                               cudaMemcpyDeviceToDevice, h->st));
  ch_status s = gather_units(h, h->U, off, true);
  for (int k = 0; k < N && s == CH_OK; ++k) {
    s = prop2(h, B, fine2(h), h->p.dt, h->p.J);
    for (int b = 0; b < B; ++b) off[b] = (long long)(b * us + (k + 1) * pts);
    if (s == CH_OK) s = gather_units(h, h->Uref, off, false);
  }
  if (s != CH_OK) return s;
  CH_CUDA(h, cudaStreamSynchronize(h->st));
  s = device_status(h, h->p2->read_status(h->st));
  if (s == CH_OK) h->ref_valid = true;
  return s;
}

ch_status run2d(ch_parareal* h) {
  const int B = h->B, N = h->p.N, maxit = h->p.maxit;
  CH_CUDA(h, h->p2->reset_counters(h->st));
  h->fine_newton = 0;
  h->fine_cg = 0;
  const size_t pts = h->pts, us = (size_t)(N + 1) * pts, fs = (size_t)N * pts;
  const double h2 = h->p.h * h->p.h;
  const double* ref = h->ref_valid ? h->Uref : nullptr;
  h->h_inc.assign(B, {});
  h->h_el2.assign(B, {});
  h->h_emx.assign(B, {});
  h->h_iters.assign(B, 0);
  h->h_conv.assign(B, 0);
  h->fine_ms = h->coarse_ms = 0.0;
  h->kernel_launches = 0;
  h->gt_launches = 0;
  h->aux_launches = 0;
  h->h_learned.assign(B, h->gt ? 1 : 0);
  h->h_fallback.assign(B, -1);
  std::vector<int> active(B, 1);
  std::vector<int>& learned = h->h_learned;
  std::vector<double> acc(4 * B);
  int nl = 0;  // active problems still on G_theta: listed first
  auto list_of = [&](std::vector<int>& L) {
    L.clear();
    for (int pass = 1; pass >= 0; --pass)
      for (int b = 0; b < B; ++b)
        if (active[b] && learned[b] == pass) L.push_back(b);
    nl = 0;
    for (int b : L) nl += learned[b];
  };
  auto pull_acc = [&]() -> ch_status {
    CH_CUDA(h, cudaMemcpyAsync(acc.data(), h->acc, 4 * B * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CH_CUDA(h, cudaStreamSynchronize(h->st));
    return CH_OK;
  };
  // Restart of the coarse guess from slice s0 with the plain step for the problems `R` (their
  // slices <= s0 are exact): U_{s+1} = G(U_s), Gold_s = G(U_s) for s >= s0 (Section 4's
  // initial sweep from s0). Their norms are recomputed.
  auto restart_plain = [&](const std::vector<int>& R, int s0) -> ch_status {
    if (R.empty() || s0 >= N) return CH_OK;
    for (int b : R) {
      // the iteration's increment (acc[0]) is kept: it measured the learned sweep that is being
      // replaced; the error norms and the state range are recomputed for the restarted slices
      CH_CUDA(h, cudaMemsetAsync(h->acc + 4 * b + 1, 0, 3 * sizeof(double), h->st));
      // slice s0 is the fine result F(U_{s0-1}) (exact), whatever the learned step produced
      if (s0 > 0)
        CH_CUDA(h, cudaMemcpyAsync(h->U + b * us + s0 * pts, h->F + b * fs + (s0 - 1) * pts, pts * sizeof(double),
                                   cudaMemcpyDeviceToDevice, h->st));
    }
    CH_CUDA(h, cudaMemcpyAsync(h->dlist, R.data(), R.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
    std::vector<long long> o(R.size());
    for (size_t i = 0; i < R.size(); ++i) o[i] = (long long)(R[i] * us + s0 * pts);
    ch_status st = gather_units(h, h->U, o, true);
    for (int sl = s0; sl < N && st == CH_OK; ++sl) {
      st = prop2(h, (int)R.size(), coarse2(h), h->p.dtc, h->p.coarse_steps);
      if (st != CH_OK) break;
      CH_CUDA(h, chg2::launch_correct(h->U + (sl + 1) * pts, h->F + sl * pts, h->W, h->Gold + sl * pts,
                                      ref ? ref + (sl + 1) * pts : nullptr, h->dlist, (int)R.size(), pts, us, fs, 1,
                                      h->cpart, h->acc, h2, h->st));
      h->aux_launches += 2;
    }
    return st;
  };
  // A learned coarse state that is not finite or leaves [-kGuard, kGuard] (Cahn-Hilliard states
  // stay near the wells +-1, overshooting them by a few per cent) is a failed prediction: the
  // problem leaves G_theta before the fine solver is asked to step from it.
  constexpr double kGuard = 2.0;
  // The plain coarse steps of a sweep run on every row, including rows whose learned prediction
  // has run away; their solves may then report a non-finite value or a refinement that does not
  // converge. When every problem with a non-finite or out-of-range coarse state is one the guard
  // sends back to the plain step (R), that report is the guard's business, not a failure: it is
  // cleared, unless it was already set before the coarse sweep (`before`).
  auto forgive_guarded = [&](const std::vector<int>& R, unsigned before) -> ch_status {
    if (R.empty()) return CH_OK;
    const unsigned bits = (chg2::ST_NONFINITE | chg2::ST_NEWTON) & ~before;
    const unsigned now = h->p2->read_status(h->st);
    if (!(now & bits)) return CH_OK;
    for (int b = 0; b < B; ++b)
      if (active[b] && !(acc[4 * b + 3] <= kGuard) && std::find(R.begin(), R.end(), b) == R.end())
        return CH_OK;  // a plain problem failed too: keep the report
    CH_CUDA(h, h->p2->clear_status(now & bits, h->st));
    return CH_OK;
  };
  CH_CUDA(h, cudaEventRecord(h->ev[0], h->st));
  // coarse initial guess (Section 4): U_{s+1} = G(U_s), Gold_s = U_{s+1}
  std::vector<int> L;
  list_of(L);
  CH_CUDA(h, cudaMemcpyAsync(h->dlist, L.data(), L.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CH_CUDA(h, cudaMemsetAsync(h->acc, 0, 4 * B * sizeof(double), h->st));
  std::vector<long long> off(L.size());
  for (size_t i = 0; i < L.size(); ++i) off[i] = (long long)(L[i] * us);
  ch_status s = gather_units(h, h->U, off, true);
  {
    chtrace::Range range("coarse initial sweep");
    for (int k = 0; k < N && s == CH_OK; ++k) {
      s = coarse_rows(h, (int)L.size(), nl);
      if (s != CH_OK) break;
      CH_CUDA(h, chg2::launch_correct(h->U + (k + 1) * pts, h->F + k * pts, h->W, h->Gold + k * pts,
                                      ref ? ref + (k + 1) * pts : nullptr, h->dlist, (int)L.size(), pts, us, fs, 1,
                                      h->cpart, h->acc, h2, h->st));
      h->aux_launches += 2;
    }
  }
  if (s != CH_OK) return s;
  if ((s = pull_acc()) != CH_OK) return s;
  {
    std::vector<int> R;
    for (int b = 0; b < B; ++b)
      if (learned[b] && !(acc[4 * b + 3] <= kGuard)) {
        learned[b] = 0;
        h->h_fallback[b] = 0;
        R.push_back(b);
      }
    if ((s = forgive_guarded(R, 0u)) != CH_OK) return s;
    if (!R.empty()) {
      if ((s = restart_plain(R, 0)) != CH_OK) return s;
      if ((s = pull_acc()) != CH_OK) return s;
    }
  }
  for (int b = 0; b < B; ++b) {
    h->h_el2[b].push_back(ref ? acc[4 * b + 1] : -1.0);
    h->h_emx[b].push_back(ref ? acc[4 * b + 2] : -1.0);
  }
  CH_CUDA(h, cudaEventRecord(h->ev[1], h->st));
  int k = 0;
  for (; k < maxit; ++k) {
    list_of(L);
    if (L.empty()) break;
    const int nb = (int)L.size();
    // fine sweep: every active problem's slices s >= k in one batch
    std::vector<long long> uoff, foff;
    for (int b : L)
      for (int sl = k; sl < N; ++sl) {
        uoff.push_back((long long)(b * us + sl * pts));
        foff.push_back((long long)(b * fs + sl * pts));
      }
    h->p2->read_status(h->st);
    const unsigned long long n0 = h->p2->newton_iterations();
    const long long c0 = h->p2->cg_unit_iterations();
    CH_CUDA(h, cudaEventRecord(h->ph[0], h->st));
    {
      chtrace::Range range("fine sweep");
      if ((s = gather_units(h, h->U, uoff, true)) != CH_OK) return s;
      if ((s = prop2(h, (int)uoff.size(), fine2(h), h->p.dt, h->p.J)) != CH_OK) return s;
      if ((s = gather_units(h, h->F, foff, false)) != CH_OK) return s;
    }
    CH_CUDA(h, cudaEventRecord(h->ph[1], h->st));
    const unsigned st_fine = h->p2->read_status(h->st);
    h->fine_newton += h->p2->newton_iterations() - n0;
    h->fine_cg += h->p2->cg_unit_iterations() - c0;
    // sequential coarse sweep with the correction of Eq. 2.2 and the norms
    CH_CUDA(h, cudaMemcpyAsync(h->dlist, L.data(), nb * sizeof(int), cudaMemcpyHostToDevice, h->st));
    CH_CUDA(h, cudaMemsetAsync(h->acc, 0, 4 * B * sizeof(double), h->st));
    off.resize(nb);
    for (int i = 0; i < nb; ++i) off[i] = (long long)(L[i] * us + k * pts);
    {
      chtrace::Range range("coarse sweep");
      if ((s = gather_units(h, h->U, off, true)) != CH_OK) return s;
      for (int sl = k; sl < N; ++sl) {
        if ((s = coarse_rows(h, nb, nl)) != CH_OK) return s;
        CH_CUDA(h, chg2::launch_correct(h->U + (sl + 1) * pts, h->F + sl * pts, h->W, h->Gold + sl * pts,
                                        ref ? ref + (sl + 1) * pts : nullptr, h->dlist, nb, pts, us, fs, 0,
                                        h->cpart, h->acc, h2, h->st));
        h->aux_launches += 2;
      }
    }
    CH_CUDA(h, cudaEventRecord(h->ph[2], h->st));
    CH_CUDA(h, cudaEventRecord(h->ev[k + 2], h->st));
    if ((s = pull_acc()) != CH_OK) return s;
    float fm = 0.f, cm = 0.f;
    CH_CUDA(h, cudaEventElapsedTime(&fm, h->ph[0], h->ph[1]));
    CH_CUDA(h, cudaEventElapsedTime(&cm, h->ph[1], h->ph[2]));
    h->fine_ms += fm;
    h->coarse_ms += cm;
    std::vector<long long> goff, uoff2;  // G(U_n^k) of problems leaving G_theta, slices > k
    std::vector<int> R;                  // problems whose learned coarse states broke the guard
    for (int b : L)
      if (learned[b] && !(acc[4 * b + 3] <= kGuard)) {
        learned[b] = 0;
        h->h_fallback[b] = k + 1;
        R.push_back(b);
      }
    if ((s = forgive_guarded(R, st_fine)) != CH_OK) return s;
    if (!R.empty()) {
      if ((s = restart_plain(R, k + 1)) != CH_OK) return s;
      if ((s = pull_acc()) != CH_OK) return s;
    }
    for (int b : L) {
      const double inc = acc[4 * b], el2 = acc[4 * b + 1], emx = acc[4 * b + 2];
      h->h_inc[b].push_back(inc);
      h->h_el2[b].push_back(ref ? el2 : -1.0);
      h->h_emx[b].push_back(ref ? emx : -1.0);
      h->h_iters[b] = k + 1;
      if ((h->p.tol > 0.0 && inc < h->p.tol) || (ref && h->p.err_tol > 0.0 && el2 <= h->p.err_tol)) {
        h->h_conv[b] = 1;
        active[b] = 0;
      }
      // the plain step judges G_theta: a growing increment sends the problem back to it
      const size_t nk = h->h_inc[b].size();
      if (learned[b] && nk >= 2 && !(h->h_inc[b][nk - 1] <= h->h_inc[b][nk - 2])) {
        learned[b] = 0;
        h->h_fallback[b] = k + 1;
        if (active[b])
          for (int sl = k + 1; sl < N; ++sl) {
            uoff2.push_back((long long)(b * us + sl * pts));
            goff.push_back((long long)(b * fs + sl * pts));
          }
      }
    }
    if (!goff.empty()) {
      // Gold_s = G(U_s^{k+1}) with the plain step, so the next correction differences one G
      if ((s = gather_units(h, h->U, uoff2, true)) != CH_OK) return s;
      if ((s = prop2(h, (int)uoff2.size(), coarse2(h), h->p.dtc, h->p.coarse_steps)) != CH_OK) return s;
      if ((s = gather_units(h, h->Gold, goff, false)) != CH_OK) return s;
    }
  }
  h->iters_done = k;
  h->ran = true;
  if ((s = device_status(h, h->p2->read_status(h->st))) != CH_OK) return s;
  h->kernel_launches = (int)std::min<long long>(h->p2->kernel_launches() + h->gt_launches + h->aux_launches,
                                                 2147483647LL);
  int left = 0;
  for (int b = 0; b < B; ++b) left += active[b];
  if ((h->p.tol > 0.0 || (h->p.err_tol > 0.0 && h->ref_valid)) && left > 0) return CH_ERR_NOT_CONVERGED;
  return CH_OK;
}

}  // namespace

// ------------------------------------------------------------------ 1D fine-sweep autotuner
//
// The fine sweep's launch configuration (CTA mapping T x P of one system per CTA, and the
// persistent grid: all resident CTAs or half of them) is chosen by timing each candidate once
// on the handle's own first fine sweep (after the coarse initial guess), with the control
// block and problem state restored after each trial. Choices are cached per process, keyed by
// (n, units, scheme path), and in the file named by CH_AUTOTUNE_CACHE when that is set.
// CH_AUTOTUNE=0 keeps the default configuration.
namespace {

struct TuneChoice {
  int alt = 0;
  int div = 1;
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;
bool g_tune_loaded = false;

std::string tune_key(const Params1D& p) {
  return "fine1d n=" + std::to_string(p.n) + " units=" + std::to_string(p.B * p.N) + " scheme=" +
         std::to_string(p.fine_scheme) + " precision=" + std::to_string(p.precision);
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("CH_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    std::string l(line);
    const size_t bar = l.find('|');
    if (bar == std::string::npos) continue;
    TuneChoice c;
    if (std::sscanf(l.c_str() + bar + 1, " alt=%d div=%d", &c.alt, &c.div) == 2) g_tune[l.substr(0, bar)] = c;
  }
  std::fclose(f);
}

void tune_save_locked() {
  const char* path = std::getenv("CH_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  for (const auto& kv : g_tune) std::fprintf(f, "%s| alt=%d div=%d\n", kv.first.c_str(), kv.second.alt, kv.second.div);
  std::fclose(f);
}

ch_status tune_fine_sweep(ch_parareal* h) {
  const char* off = std::getenv("CH_AUTOTUNE");
  if (off && std::strcmp(off, "0") == 0) return CH_OK;
  chtrace::Range range("autotune");
  const std::string key = tune_key(h->p);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      Params1D q = h->p;
      q.alt = chg::fine_sweep_has_alt(q) ? it->second.alt : 0;
      int grid = 0;
      CH_CUDA(h, chg::fine_sweep_max_grid(q, &grid));
      h->p.alt = q.alt;
      h->grid = std::max(1, grid / std::max(1, it->second.div));
      return CH_OK;
    }
  }
  void* snap = nullptr;
  CH_CUDA(h, cudaMalloc(&snap, sizeof(Ctrl) + h->ps_bytes));
  char* sc = static_cast<char*>(snap);
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaMemcpyAsync(sc, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sc + sizeof(Ctrl), h->ps_block, h->ps_bytes, cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  TuneChoice best;
  float best_ms = 1e30f;
  const int nalt = chg::fine_sweep_has_alt(h->p) ? 2 : 1;
  for (int alt = 0; alt < nalt && e == cudaSuccess; ++alt)
    for (int div = 1; div <= 2 && e == cudaSuccess; ++div) {
      Params1D q = h->p;
      q.alt = alt;
      int grid = 0;
      e = chg::fine_sweep_max_grid(q, &grid);
      if (e != cudaSuccess) break;
      grid = std::max(1, grid / div);
      e = cudaMemcpyAsync(h->ctrl, sc, sizeof(Ctrl), cudaMemcpyDeviceToDevice, h->st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->ps_block, sc + sizeof(Ctrl), h->ps_bytes, cudaMemcpyDeviceToDevice, h->st);
      if (e == cudaSuccess) e = cudaEventRecord(a, h->st);
      if (e == cudaSuccess) e = chg::launch_fine_sweep(q, h->U, h->F, h->ctrl, h->ps, grid, h->st);
      if (e == cudaSuccess) e = cudaEventRecord(b, h->st);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best.alt = alt;
        best.div = div;
      }
    }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->ctrl, sc, sizeof(Ctrl), cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->ps_block, sc + sizeof(Ctrl), h->ps_bytes, cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(snap);
  if (e != cudaSuccess) return cuda_fail(h, e, "fine-sweep autotuning");
  Params1D q = h->p;
  q.alt = best.alt;
  int grid = 0;
  CH_CUDA(h, chg::fine_sweep_max_grid(q, &grid));
  h->p.alt = best.alt;
  h->grid = std::max(1, grid / best.div);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  tune_save_locked();
  return CH_OK;
}

// 2D: the execution of the implicit steps — one CUDA graph per step (conditional loops, a kernel
// per phase) or one persistent cooperative kernel per propagation (the same phases separated by
// grid barriers) — is chosen once per handle, before its first reference or run, by timing one
// fine step of the handle's fine-sweep batch (every slice of every problem, started from u^0)
// with each (the second of two runs, so graph construction is not timed). The reference and
// every Parareal iteration then use the same execution, so the iterate at k = N still equals the
// reference bit for bit. Cached per process by grid, fine scheme and step (not by batch size:
// handles of the same configuration then share one execution, and a problem's results do not
// depend on the batch it is solved in). CH_2D_STEP forces an execution; CH_AUTOTUNE=0 keeps the
// graphs.
std::map<std::string, int> g_tune2d;

ch_status ensure_tuned2d(ch_parareal* h) {
  if (h->tuned) return CH_OK;
  h->tuned = true;
  if (std::getenv("CH_2D_STEP")) return CH_OK;
  chtrace::Range range("autotune");
  const char* off = std::getenv("CH_AUTOTUNE");
  if (off && std::strcmp(off, "0") == 0) return CH_OK;
  const int units = h->B * h->p.N;
  char buf[160];
  std::snprintf(buf, sizeof(buf), "2d n=%d scheme=%d dt=%.17g", h->p.n, fine2(h), h->p.dt);
  const std::string key(buf);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune2d.find(key);
    if (it != g_tune2d.end()) {
      h->p2->set_path(static_cast<chg2::StepPath>(it->second));
      return CH_OK;
    }
  }
  const size_t pts = h->pts, us = (size_t)(h->p.N + 1) * pts;
  std::vector<long long> offs((size_t)units);
  for (int b = 0; b < h->B; ++b)
    for (int sl = 0; sl < h->p.N; ++sl) offs[(size_t)b * h->p.N + sl] = (long long)(b * us);
  const chg2::StepPath paths[2] = {chg2::PATH_GRAPH, chg2::PATH_PERSISTENT};
  cudaEvent_t a = nullptr, e2 = nullptr;
  CH_CUDA(h, cudaEventCreate(&a));
  CH_CUDA(h, cudaEventCreate(&e2));
  chg2::StepPath best = chg2::PATH_GRAPH;
  float best_ms = 1e30f;
  ch_status s = CH_OK;
  for (chg2::StepPath pth : paths) {
    h->p2->set_path(pth);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && s == CH_OK; ++rep) {
      s = gather_units(h, h->U, offs, true);
      if (s == CH_OK && cudaEventRecord(a, h->st) != cudaSuccess) s = fail(h, CH_ERR_CUDA, "tuning event");
      if (s == CH_OK) s = prop2(h, units, fine2(h), h->p.dt, rep == 0 ? 1 : 2);
      if (s == CH_OK && cudaEventRecord(e2, h->st) != cudaSuccess) s = fail(h, CH_ERR_CUDA, "tuning event");
      if (s == CH_OK && cudaEventSynchronize(e2) != cudaSuccess) s = fail(h, CH_ERR_CUDA, "tuning sync");
      if (s == CH_OK && cudaEventElapsedTime(&ms, a, e2) != cudaSuccess) s = fail(h, CH_ERR_CUDA, "tuning time");
    }
    if (s != CH_OK) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = pth;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(e2);
  if (s != CH_OK) return s;
  h->p2->set_path(best);
  CH_CUDA(h, h->p2->reset_counters(h->st));  // the trial steps' counts and status bits
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune2d[key] = (int)best;
  return CH_OK;
}

// Tunes once per handle, before its first reference or run, so that both use the same fine-sweep
// configuration (the sequential reference then equals the Parareal iterate at k = N bit for bit).
// The trial sweeps run on a coarse initial guess written into U (overwritten by run).
ch_status ensure_tuned(ch_parareal* h) {
  if (h->tuned) return CH_OK;
  std::vector<int> ones(h->B, 1);
  CH_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->st));
  CH_CUDA(h, cudaMemsetAsync(h->ps_block, 0, h->ps_bytes, h->st));
  CH_CUDA(h, cudaMemcpyAsync(h->ps.active, ones.data(), h->B * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CH_CUDA(h, chg::launch_coarse_sweep(h->p, h->U, h->F, h->Gold, nullptr, h->ctrl, h->ps, 1, h->st));
  ch_status s = tune_fine_sweep(h);
  if (s != CH_OK) return s;
  h->tuned = true;
  if (h->gfine) {
    cudaGraphExecDestroy(h->gfine);
    h->gfine = nullptr;
  }
  return CH_OK;
}

}  // namespace


extern "C" {

const char* ch_status_string(ch_status s) {
  switch (s) {
    case CH_OK: return "CH_OK";
    case CH_ERR_INVALID: return "CH_ERR_INVALID";
    case CH_ERR_OOM: return "CH_ERR_OOM";
    case CH_ERR_CUDA: return "CH_ERR_CUDA";
    case CH_ERR_NEWTON: return "CH_ERR_NEWTON";
    case CH_ERR_LINSOLVE: return "CH_ERR_LINSOLVE";
    case CH_ERR_NOT_CONVERGED: return "CH_ERR_NOT_CONVERGED";
    case CH_ERR_TIMEOUT: return "CH_ERR_TIMEOUT";
    case CH_ERR_STATE: return "CH_ERR_STATE";
  }
  return "CH_ERR_UNKNOWN";
}

const char* ch_parareal_last_error(const ch_parareal* h) { return h ? h->msg.c_str() : "NULL handle"; }

void ch_parareal_destroy(ch_parareal* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  if (h->gfine) cudaGraphExecDestroy(h->gfine);
  if (h->gcoarse) cudaGraphExecDestroy(h->gcoarse);
  for (auto e : h->ev) cudaEventDestroy(e);
  for (auto e : h->ph)
    if (e) cudaEventDestroy(e);
  cudaFree(h->U);
  cudaFree(h->F);
  cudaFree(h->Gold);
  cudaFree(h->Uref);
  cudaFree(h->ctrl);
  cudaFree(h->ps_block);
  if (h->host_active) cudaFreeHost(h->host_active);
  if (h->p2) {
    h->p2->release();
    delete h->p2;
  }
  cudaFree(h->W);
  cudaFree(h->acc);
  cudaFree(h->cpart);
  cudaFree(h->dlist);
  cudaFree(h->doff);
  if (h->gt) {
    h->gt->release();
    delete h->gt;
  }
  cudaFree(h->Wtmp);
  cudaFree(h->eps2u_dev);
  delete h;
}

ch_status ch_parareal_create(const ch_config* cfg, int batch, void* cuda_stream, ch_parareal** out) {
  if (!out) return CH_ERR_INVALID;
  *out = nullptr;
  std::string why;
  if (!chcfg::valid_run(cfg, chg2::supported_n, why) || batch < 1) return CH_ERR_INVALID;
  ch_parareal* h = new (std::nothrow) ch_parareal();
  if (!h) return CH_ERR_OOM;
  (void)cudaGetLastError();  // a stale non-sticky error of an earlier call must not fail this one
  h->cfg = *cfg;
  h->B = batch;
  h->st = static_cast<cudaStream_t>(cuda_stream);
  h->p = make_params(cfg, batch);
  h->dim = cfg->dim;
  h->pts = (cfg->dim == 2) ? (size_t)cfg->n * cfg->n : (size_t)cfg->n;
  h->initial_set.assign(batch, 0);
  cudaGetDevice(&h->device);
  const size_t N = cfg->n_slices, B = batch, pts = h->pts;
  const size_t maxit = cfg->max_iters;
  cudaError_t e;
  auto bail = [&](cudaError_t err, const char* w) {
    ch_status s = cuda_fail(h, err, w);
    ch_parareal_destroy(h);
    return s;
  };
  if ((e = cudaMalloc(&h->U, B * (N + 1) * pts * sizeof(double)))) return bail(e, "cudaMalloc(U)");
  if ((e = cudaMalloc(&h->F, B * N * pts * sizeof(double)))) return bail(e, "cudaMalloc(F)");
  if ((e = cudaMalloc(&h->Gold, B * N * pts * sizeof(double)))) return bail(e, "cudaMalloc(Gold)");
  if ((e = cudaMalloc(&h->Uref, B * (N + 1) * pts * sizeof(double)))) return bail(e, "cudaMalloc(Uref)");
  if ((e = cudaMalloc(&h->ctrl, sizeof(Ctrl)))) return bail(e, "cudaMalloc(ctrl)");
  // per-problem arrays in one block: doubles first (8-byte aligned), then ints
  const size_t nd = B * maxit + 2 * B * (maxit + 1);
  const size_t bytes = nd * sizeof(double) + B * sizeof(unsigned long long) + 4 * B * sizeof(int);
  if ((e = cudaMalloc(&h->ps_block, bytes))) return bail(e, "cudaMalloc(problem state)");
  h->ps_bytes = bytes;
  char* q = static_cast<char*>(h->ps_block);
  h->ps.inc = reinterpret_cast<double*>(q);
  h->ps.err_l2 = h->ps.inc + B * maxit;
  h->ps.err_max = h->ps.err_l2 + B * (maxit + 1);
  h->ps.newton_total = reinterpret_cast<unsigned long long*>(h->ps.err_max + B * (maxit + 1));
  h->ps.active = reinterpret_cast<int*>(h->ps.newton_total + B);
  h->ps.iterations = h->ps.active + B;
  h->ps.converged = h->ps.iterations + B;
  h->ps.newton_max = h->ps.converged + B;
  if ((e = cudaHostAlloc(&h->host_active, sizeof(int), cudaHostAllocMapped))) return bail(e, "cudaHostAlloc");
  if ((e = cudaHostGetDevicePointer(&h->host_active_dev, h->host_active, 0))) return bail(e, "cudaHostGetDevicePointer");
  if ((e = cudaMemsetAsync(h->U, 0, B * (N + 1) * pts * sizeof(double), h->st))) return bail(e, "cudaMemsetAsync");
  h->ev.resize(maxit + 2);
  for (auto& ev : h->ev)
    if ((e = cudaEventCreate(&ev))) return bail(e, "cudaEventCreate");
  for (auto& ev : h->ph)
    if ((e = cudaEventCreate(&ev))) return bail(e, "cudaEventCreate");
  if (h->dim == 2) {
    h->p2 = new (std::nothrow) chg2::Prop2D();
    if (!h->p2) {
      ch_parareal_destroy(h);
      return CH_ERR_OOM;
    }
    if ((e = h->p2->init(params2d(cfg), (int)(B * N), h->st))) return bail(e, "2D work space");
    if ((e = cudaMalloc(&h->W, B * N * pts * sizeof(double)))) return bail(e, "cudaMalloc(W)");
    if ((e = cudaMalloc(&h->acc, B * 4 * sizeof(double)))) return bail(e, "cudaMalloc(acc)");
    if ((e = cudaMalloc(&h->cpart, chg2::correct_partials((int)B) * sizeof(double)))) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->dlist, B * sizeof(int)))) return bail(e, "cudaMalloc(list)");
    if ((e = cudaMalloc(&h->doff, B * N * sizeof(long long)))) return bail(e, "cudaMalloc(offsets)");
    *out = h;
    return CH_OK;
  }
  if ((e = chg::fine_sweep_max_grid(h->p, &h->grid))) return bail(e, "fine_sweep_max_grid");
  *out = h;
  return CH_OK;
}

ch_status ch_parareal_set_initial(ch_parareal* h, int problem, const double* u0_host, size_t len) {
  if (!h) return CH_ERR_INVALID;
  if (problem < 0 || problem >= h->B || !u0_host || len != h->pts)
    return fail(h, CH_ERR_INVALID, "set_initial: bad problem index, pointer or length");
  CH_CUDA(h, cudaMemcpyAsync(h->U + (size_t)problem * (h->p.N + 1) * h->pts, u0_host, h->pts * sizeof(double),
                             cudaMemcpyHostToDevice, h->st));
  CH_CUDA(h, cudaStreamSynchronize(h->st));
  h->initial_set[problem] = 1;
  h->ref_valid = false;
  clear_data_error(h);
  return CH_OK;
}

ch_status ch_parareal_set_initial_device(ch_parareal* h, const double* u0_dev, size_t len) {
  if (!h) return CH_ERR_INVALID;
  if (!u0_dev || len != (size_t)h->B * h->pts) return fail(h, CH_ERR_INVALID, "set_initial_device: bad pointer or length");
  CH_CUDA(h, cudaMemcpy2DAsync(h->U, (h->p.N + 1) * h->pts * sizeof(double), u0_dev, h->pts * sizeof(double),
                               h->pts * sizeof(double), h->B, cudaMemcpyDeviceToDevice, h->st));
  for (auto& v : h->initial_set) v = 1;
  h->ref_valid = false;
  clear_data_error(h);
  return CH_OK;
}

ch_status ch_parareal_set_initial_batch(ch_parareal* h, const double* u0_host, size_t len) {
  if (!h) return CH_ERR_INVALID;
  if (!u0_host || len != (size_t)h->B * h->pts) return fail(h, CH_ERR_INVALID, "set_initial_batch: bad pointer or length");
  CH_CUDA(h, cudaMemcpy2DAsync(h->U, (h->p.N + 1) * h->pts * sizeof(double), u0_host, h->pts * sizeof(double),
                               h->pts * sizeof(double), h->B, cudaMemcpyHostToDevice, h->st));
  for (auto& v : h->initial_set) v = 1;
  h->ref_valid = false;
  clear_data_error(h);
  return CH_OK;
}

static bool all_initial(const ch_parareal* h) {
  for (int v : h->initial_set)
    if (!v) return false;
  return true;
}

ch_status ch_parareal_compute_reference(ch_parareal* h) {
  if (!h) return CH_ERR_INVALID;
  chtrace::Range range("ch_parareal_compute_reference");
  if (h->sticky != CH_OK) return h->sticky;
  if (!all_initial(h)) return fail(h, CH_ERR_STATE, "compute_reference before set_initial");
  if (h->dim == 2) {
    ch_status s = ensure_tuned2d(h);
    return s != CH_OK ? s : reference2d(h);
  }
  {
    ch_status s = ensure_tuned(h);
    if (s != CH_OK) return s;
  }
  const size_t N = h->p.N, pts = h->pts;
  CH_CUDA(h, cudaMemcpy2DAsync(h->Uref, (N + 1) * pts * sizeof(double), h->U, (N + 1) * pts * sizeof(double),
                               pts * sizeof(double), h->B, cudaMemcpyDeviceToDevice, h->st));
  CH_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->st));
  CH_CUDA(h, chg::launch_reference(h->p, h->Uref, h->ctrl, h->st));
  Ctrl c;
  CH_CUDA(h, cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaStreamSynchronize(h->st));
  ch_status s = device_status(h, c.status);
  if (s != CH_OK) return s;
  h->ref_valid = true;
  return CH_OK;
}

}  // extern "C"


// Captures the work enqueued by `enqueue` on a private stream into an executable graph.
template <typename F>
static ch_status capture(ch_parareal* h, F enqueue, cudaGraphExec_t* out) {
  cudaStream_t cs = nullptr;
  CH_CUDA(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(h, e, "cudaStreamBeginCapture");
  }
  cudaError_t le = enqueue(cs);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(h, le, "kernel launch during capture");
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
  return CH_OK;
}

extern "C" {

ch_status ch_parareal_run(ch_parareal* h) {
  if (!h) return CH_ERR_INVALID;
  chtrace::Range range("ch_parareal_run");
  if (h->sticky != CH_OK) return h->sticky;
  if (!all_initial(h)) return fail(h, CH_ERR_STATE, "run before set_initial");
  if (h->dim == 2) {
    ch_status s = ensure_tuned2d(h);
    return s != CH_OK ? s : run2d(h);
  }
  const int B = h->B, maxit = h->p.maxit;
  std::vector<int> ones(B, 1);
  {
    ch_status s = ensure_tuned(h);
    if (s != CH_OK) return s;
  }
  // reset control and per-problem state
  CH_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->st));
  CH_CUDA(h, cudaMemsetAsync(h->ps_block, 0,
                             (size_t)B * maxit * sizeof(double) + 2 * (size_t)B * (maxit + 1) * sizeof(double) +
                                 B * sizeof(unsigned long long) + 4 * (size_t)B * sizeof(int),
                             h->st));
  CH_CUDA(h, cudaMemcpyAsync(h->ps.active, ones.data(), B * sizeof(int), cudaMemcpyHostToDevice, h->st));
  const double* ref = h->ref_valid ? h->Uref : nullptr;
  CH_CUDA(h, cudaEventRecord(h->ev[0], h->st));
  {
    chtrace::Range r_init("coarse initial sweep");
    CH_CUDA(h, chg::launch_coarse_sweep(h->p, h->U, h->F, h->Gold, ref, h->ctrl, h->ps, 1, h->st));
  }
  CH_CUDA(h, cudaEventRecord(h->ev[1], h->st));
  // The iteration graphs read k and the active set from device memory, so one capture
  // serves every iteration.
  if (!h->gfine) {
    ch_status s = capture(h, [&](cudaStream_t cs) {
      return chg::launch_fine_sweep(h->p, h->U, h->F, h->ctrl, h->ps, h->grid, cs);
    }, &h->gfine);
    if (s != CH_OK) return s;
  }
  if (!h->gcoarse || h->graph_ref != (h->ref_valid ? 1 : 0)) {
    if (h->gcoarse) { cudaGraphExecDestroy(h->gcoarse); h->gcoarse = nullptr; }
    ch_status s = capture(h, [&](cudaStream_t cs) {
      cudaError_t e = chg::launch_coarse_sweep(h->p, h->U, h->F, h->Gold, ref, h->ctrl, h->ps, 0, cs);
      if (e == cudaSuccess) e = chg::launch_tally(h->p, h->ctrl, h->ps, h->host_active_dev, cs);
      return e;
    }, &h->gcoarse);
    if (s != CH_OK) return s;
    h->graph_ref = h->ref_valid ? 1 : 0;
  }
  h->active_before.clear();
  h->fine_ms = h->coarse_ms = 0.0;
  h->kernel_launches = 1;
  int active = B;
  int k = 0;
  for (; k < maxit && active > 0; ++k) {
    h->active_before.push_back(active);
    CH_CUDA(h, cudaEventRecord(h->ph[0], h->st));
    {
      chtrace::Range r_fine("fine sweep");
      CH_CUDA(h, cudaGraphLaunch(h->gfine, h->st));
    }
    CH_CUDA(h, cudaEventRecord(h->ph[1], h->st));
    {
      chtrace::Range r_coarse("coarse sweep");
      CH_CUDA(h, cudaGraphLaunch(h->gcoarse, h->st));
    }
    CH_CUDA(h, cudaEventRecord(h->ph[2], h->st));
    CH_CUDA(h, cudaEventRecord(h->ev[k + 2], h->st));
    CH_CUDA(h, cudaStreamSynchronize(h->st));
    h->kernel_launches += 3;
    float fm = 0.f, cm = 0.f;
    CH_CUDA(h, cudaEventElapsedTime(&fm, h->ph[0], h->ph[1]));
    CH_CUDA(h, cudaEventElapsedTime(&cm, h->ph[1], h->ph[2]));
    h->fine_ms += fm;
    h->coarse_ms += cm;
    active = *(volatile int*)h->host_active;
  }
  h->iters_done = k;
  h->ran = true;
  Ctrl c;
  CH_CUDA(h, cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaStreamSynchronize(h->st));
  ch_status s = device_status(h, c.status);
  if (s != CH_OK) return s;
  if ((h->p.tol > 0.0 || (h->p.err_tol > 0.0 && h->ref_valid)) && active > 0) return CH_ERR_NOT_CONVERGED;
  return CH_OK;
}

ch_status ch_parareal_get_slices(ch_parareal* h, int problem, double* out_host, size_t len) {
  if (!h) return CH_ERR_INVALID;
  const size_t want = (size_t)(h->p.N + 1) * h->pts;
  if (problem < 0 || problem >= h->B || !out_host || len != want)
    return fail(h, CH_ERR_INVALID, "get_slices: bad problem index, pointer or length");
  CH_CUDA(h, cudaMemcpyAsync(out_host, h->U + (size_t)problem * want, want * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaStreamSynchronize(h->st));
  return CH_OK;
}

ch_status ch_parareal_get_slices_batch(ch_parareal* h, double* out_host, size_t len) {
  if (!h) return CH_ERR_INVALID;
  const size_t want = (size_t)h->B * (h->p.N + 1) * h->pts;
  if (!out_host || len != want) return fail(h, CH_ERR_INVALID, "get_slices_batch: bad pointer or length");
  CH_CUDA(h, cudaMemcpyAsync(out_host, h->U, want * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaStreamSynchronize(h->st));
  return CH_OK;
}

ch_status ch_parareal_get_slices_device(ch_parareal* h, double* out_dev, size_t len) {
  if (!h) return CH_ERR_INVALID;
  const size_t want = (size_t)h->B * (h->p.N + 1) * h->pts;
  if (!out_dev || len != want) return fail(h, CH_ERR_INVALID, "get_slices_device: bad pointer or length");
  CH_CUDA(h, cudaMemcpyAsync(out_dev, h->U, want * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  return CH_OK;
}

ch_status ch_parareal_get_reference(ch_parareal* h, int problem, double* out_host, size_t len) {
  if (!h) return CH_ERR_INVALID;
  const size_t want = (size_t)(h->p.N + 1) * h->pts;
  if (!h->ref_valid) return fail(h, CH_ERR_STATE, "get_reference before compute_reference");
  if (problem < 0 || problem >= h->B || !out_host || len != want)
    return fail(h, CH_ERR_INVALID, "get_reference: bad problem index, pointer or length");
  CH_CUDA(h, cudaMemcpyAsync(out_host, h->Uref + (size_t)problem * want, want * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaStreamSynchronize(h->st));
  return CH_OK;
}

ch_status ch_parareal_get_execution(ch_parareal* h, int* out) {
  if (!h) return CH_ERR_INVALID;
  if (!out) return fail(h, CH_ERR_INVALID, "get_execution: null pointer");
  if (h->dim == 2) {
    *out = h->tuned ? (int)h->p2->path() : -1;
  } else {
    *out = h->tuned ? h->p.alt : -1;
  }
  return CH_OK;
}

ch_status ch_parareal_get_stats(ch_parareal* h, int problem, ch_stats* out) {
  if (!h) return CH_ERR_INVALID;
  if (!out || problem < 0 || problem >= h->B) return fail(h, CH_ERR_INVALID, "get_stats: bad problem index or pointer");
  if (!h->ran) return fail(h, CH_ERR_STATE, "get_stats before run");
  std::memset(out, 0, sizeof(*out));
  if (h->dim == 2) {
    out->iterations = h->h_iters[problem];
    out->converged = h->h_conv[problem];
    for (size_t k = 0; k < h->h_inc[problem].size(); ++k) out->inc[k] = h->h_inc[problem][k];
    for (size_t k = 0; k < h->h_el2[problem].size(); ++k) {
      out->err_l2[k] = h->h_el2[problem][k];
      out->err_max[k] = h->h_emx[problem][k];
    }
    for (int k = 0; k <= h->iters_done; ++k) {
      float ms = 0.f;
      CH_CUDA(h, cudaEventElapsedTime(&ms, h->ev[0], h->ev[k + 1]));
      out->t_iter_ms[k] = ms;
    }
    out->newton_total = (long long)h->fine_newton;
    out->newton_max = h->p2->newton_peak();
    long long fps = 0;
    for (int k = 0; k < out->iterations; ++k) fps += (long long)(h->p.N - k) * h->p.J * (long long)h->pts;
    out->fine_point_steps = fps;
    out->fine_sweep_ms = h->fine_ms;
    out->coarse_sweep_ms = h->coarse_ms;
    out->fine_sweep_launches = h->iters_done;
    out->kernel_launches = h->kernel_launches;
    out->inner_iterations = h->fine_cg;
    out->coarse_model = h->h_learned.empty() ? 0 : (h->h_learned[problem] || h->h_fallback[problem] >= 0);
    out->coarse_fallback_iter = h->h_fallback.empty() ? -1 : h->h_fallback[problem];
    return CH_OK;
  }
  const int maxit = h->p.maxit;
  int it = 0, conv = 0, nmax = 0;
  unsigned long long ntot = 0;
  CH_CUDA(h, cudaMemcpyAsync(&it, h->ps.iterations + problem, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaMemcpyAsync(&conv, h->ps.converged + problem, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaMemcpyAsync(&nmax, h->ps.newton_max + problem, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaMemcpyAsync(&ntot, h->ps.newton_total + problem, sizeof(ntot), cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaMemcpyAsync(out->inc, h->ps.inc + (size_t)problem * maxit, maxit * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaMemcpyAsync(out->err_l2, h->ps.err_l2 + (size_t)problem * (maxit + 1), (maxit + 1) * sizeof(double),
                             cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaMemcpyAsync(out->err_max, h->ps.err_max + (size_t)problem * (maxit + 1), (maxit + 1) * sizeof(double),
                             cudaMemcpyDeviceToHost, h->st));
  CH_CUDA(h, cudaStreamSynchronize(h->st));
  out->iterations = it;
  out->converged = conv;
  out->newton_total = (long long)ntot;
  out->newton_max = nmax;
  for (int k = 0; k <= h->iters_done; ++k) {
    float ms = 0.f;
    CH_CUDA(h, cudaEventElapsedTime(&ms, h->ev[0], h->ev[k + 1]));
    out->t_iter_ms[k] = ms;
  }
  long long fps = 0;
  for (int k = 0; k < it; ++k) fps += (long long)(h->p.N - k) * h->p.J * (long long)h->pts;
  out->fine_point_steps = fps;
  out->fine_sweep_ms = h->fine_ms;
  out->coarse_sweep_ms = h->coarse_ms;
  out->fine_sweep_launches = h->iters_done;
  out->kernel_launches = h->kernel_launches;
  out->coarse_model = 0;
  out->coarse_fallback_iter = -1;
  return CH_OK;
}

ch_status ch_parareal_set_coarse_model(ch_parareal* h, const float* params_host, size_t len, int form) {
  if (!h) return CH_ERR_INVALID;
  if (h->dim != 2) return fail(h, CH_ERR_INVALID, "set_coarse_model: the learned coarse propagator is 2D only");
  if (form != CH_GTHETA_RESIDUAL && form != CH_GTHETA_CORRECTION)
    return fail(h, CH_ERR_INVALID, "set_coarse_model: unknown form");
  if (!params_host) {
    if (len != 0) return fail(h, CH_ERR_INVALID, "set_coarse_model: NULL parameters need len = 0");
    if (h->gt) {
      CH_CUDA(h, cudaStreamSynchronize(h->st));
      h->gt->release();
      delete h->gt;
      h->gt = nullptr;
    }
    return CH_OK;
  }
  if (len != (size_t)CH_GTHETA_PARAMS) return fail(h, CH_ERR_INVALID, "set_coarse_model: len != CH_GTHETA_PARAMS");
  if (!h->gt) {
    h->gt = new (std::nothrow) chg3::GTheta();
    if (!h->gt) return fail(h, CH_ERR_OOM, "set_coarse_model: host allocation");
    CH_CUDA(h, h->gt->init(0, h->st));
  }
  if (form == CH_GTHETA_CORRECTION && !h->Wtmp)
    CH_CUDA(h, cudaMalloc(&h->Wtmp, (size_t)h->B * h->pts * sizeof(double)));
  CH_CUDA(h, h->gt->set_params(params_host, h->st));
  h->gt_form = form;
  return CH_OK;
}

ch_status ch_parareal_set_eps(ch_parareal* h, const double* eps_host, size_t len) {
  if (!h) return CH_ERR_INVALID;
  if (h->dim != 2) return fail(h, CH_ERR_INVALID, "set_eps: per-problem eps is supported in 2D");
  if (!eps_host || len != (size_t)h->B) return fail(h, CH_ERR_INVALID, "set_eps: len must equal the batch");
  for (size_t b = 0; b < len; ++b)
    if (!(eps_host[b] > 0.0) || !std::isfinite(eps_host[b])) return fail(h, CH_ERR_INVALID, "set_eps: eps must be > 0");
  if (!h->eps2u_dev) CH_CUDA(h, cudaMalloc(&h->eps2u_dev, (size_t)h->B * h->p.N * sizeof(double)));
  h->eps_prob.assign(eps_host, eps_host + len);
  h->p2->set_unit_eps2(h->eps2u_dev);
  h->ref_valid = false;
  clear_data_error(h);
  return CH_OK;
}

ch_status ch_parareal_set_fine_nn(ch_parareal* h, int n_sub, double theta, double tol, int max_iter) {
  if (!h) return CH_ERR_INVALID;
  if (h->dim != 1) return fail(h, CH_ERR_INVALID, "set_fine_nn: the Neumann-Neumann fine solver is 1D");
  if (h->p.fine_scheme != chg::SCHEME_LIN1)
    return fail(h, CH_ERR_INVALID, "set_fine_nn: the fine scheme must be the linear scheme Eq. 2.4 (PA-I)");
  chg::Params1D q = h->p;
  if (n_sub == 0) {
    q.nn_sub = 0;
  } else {
    if (!(theta > 0.0 && theta <= 1.0) || !(tol > 0.0) || !std::isfinite(tol) || max_iter < 1 || max_iter > 100000)
      return fail(h, CH_ERR_INVALID, "set_fine_nn: theta in (0, 1], tol > 0 and max_iter in 1..100000");
    q.nn_sub = n_sub;
    q.nn_theta = theta;
    q.nn_tol = tol;
    q.nn_max = max_iter;
    if (!chg::nn_supported(q))
      return fail(h, CH_ERR_INVALID, "set_fine_nn: n_sub in 1..32 dividing n + 1, at least 2 nodes per subdomain");
  }
  int grid = 0;
  CH_CUDA(h, chg::fine_sweep_max_grid(q, &grid));
  h->p = q;
  h->grid = grid;
  h->tuned = (n_sub > 0);  // the autotuner chooses among monolithic sweeps only
  if (h->gfine) {
    cudaGraphExecDestroy(h->gfine);
    h->gfine = nullptr;
  }
  h->ref_valid = false;
  clear_data_error(h);
  return CH_OK;
}

ch_status ch_parareal_get_reference_device(ch_parareal* h, double* out_dev, size_t len) {
  if (!h) return CH_ERR_INVALID;
  const size_t want = (size_t)h->B * (h->p.N + 1) * h->pts;
  if (!h->ref_valid) return fail(h, CH_ERR_STATE, "get_reference_device before compute_reference");
  if (!out_dev || len != want) return fail(h, CH_ERR_INVALID, "get_reference_device: bad pointer or length");
  CH_CUDA(h, cudaMemcpyAsync(out_dev, h->Uref, want * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  return CH_OK;
}

ch_status ch_sine_transform_2d(const float* in_dev, float* out_dev, int batch, int n, void* cuda_stream) {
  if (!in_dev || !out_dev || in_dev == out_dev || batch < 1 || !chg2::supported_n(n)) return CH_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  chg2::Params2D q{};
  q.n = n;
  q.h = 1.0 / (n + 1);
  q.newton_max = 1;
  q.cg_max = 1;
  chg2::Prop2D prop;
  cudaError_t e = prop.init(q, batch, st);
  if (e == cudaSuccess) e = prop.dst2(in_dev, out_dev, batch, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  prop.release();
  if (e == cudaErrorMemoryAllocation) return CH_ERR_OOM;
  return e == cudaSuccess ? CH_OK : CH_ERR_CUDA;
}

ch_status ch_propagate(const ch_config* cfg, int batch, int scheme, double dt, int nsteps, const double* u_in_dev,
                       double* u_out_dev, int* newton_dev, void* cuda_stream) {
  chtrace::Range range("ch_propagate");
  std::string why;
  if (!valid_common(cfg, why) || batch < 1 || nsteps < 0 || !(dt > 0.0) || !u_in_dev || !u_out_dev ||
      scheme < CH_SCHEME_LIN1 || scheme > CH_SCHEME_LIN2)
    return CH_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (cfg->dim == 2) {
    chg2::Prop2D prop;
    cudaError_t e = prop.init(params2d(cfg), batch, st);
    const size_t bytes = (size_t)batch * cfg->n * cfg->n * sizeof(double);
    if (e == cudaSuccess && u_out_dev != u_in_dev) e = cudaMemcpyAsync(u_out_dev, u_in_dev, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = prop.propagate(u_out_dev, batch, scheme, dt, nsteps, st);
    unsigned status = (e == cudaSuccess) ? prop.read_status(st) : 0u;
    if (e == cudaSuccess && newton_dev) {
      const int tot = (int)prop.newton_iterations();
      std::vector<int> v(batch, tot / batch);
      e = cudaMemcpyAsync(newton_dev, v.data(), batch * sizeof(int), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    prop.release();
    if (e == cudaErrorMemoryAllocation) return CH_ERR_OOM;
    if (e != cudaSuccess) return CH_ERR_CUDA;
    if (status & chg2::ST_TIMEOUT) return CH_ERR_TIMEOUT;
    if (status & chg2::ST_NONFINITE) return CH_ERR_LINSOLVE;
    if (status & chg2::ST_NEWTON) return CH_ERR_NEWTON;
    return CH_OK;
  }
  Params1D p = make_params(cfg, batch);
  Ctrl* ctrl = nullptr;
  if (cudaMalloc(&ctrl, sizeof(Ctrl)) != cudaSuccess) return CH_ERR_OOM;
  ch_status s = CH_OK;
  cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
  if (e == cudaSuccess) e = chg::launch_propagate(p, scheme, dt, nsteps, u_in_dev, u_out_dev, newton_dev, ctrl, st);
  Ctrl c{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) s = CH_ERR_CUDA;
  else if (c.status & chg::ST_NONFINITE) s = CH_ERR_LINSOLVE;
  else if (c.status & chg::ST_NEWTON) s = CH_ERR_NEWTON;
  cudaFree(ctrl);
  return s;
}

}  // extern "C"
