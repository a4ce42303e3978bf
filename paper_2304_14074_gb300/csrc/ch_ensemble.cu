// Ensembles of 2D problems on uneven grids (declared in include/ch_parareal.h).
//
// The problems are grouped by grid size; each group is one Parareal handle (its units batched in
// every launch, per-problem eps) on a stream of its own, and run() drives the groups from one
// host thread each, so the groups' graphs and kernels overlap on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ch_parareal.h"

struct ch_ensemble {
  struct Group {
    int n = 0;
    std::vector<int> problems;  // ensemble indices, in the group's batch order
    cudaStream_t st = nullptr;
    ch_parareal* h = nullptr;
  };
  std::vector<Group> groups;
  std::vector<std::pair<int, int>> where;  // problem -> (group, index in the group)
  ch_config cfg{};
  int device = 0;
  ch_status sticky = CH_OK;
  std::string msg;
};

namespace {

ch_status efail(ch_ensemble* e, ch_status s, const std::string& m) {
  if (e && e->sticky == CH_OK) {
    e->sticky = s;
    e->msg = m;
  }
  return s;
}


// Runs f(group) for every group, each from its own host thread; returns the first error.
template <typename F>
ch_status for_groups(ch_ensemble* e, F f, ch_status ok_also) {
  std::vector<ch_status> st(e->groups.size(), CH_OK);
  std::vector<std::thread> th;
  for (size_t i = 0; i < e->groups.size(); ++i)
    th.emplace_back([&, i] {
      cudaSetDevice(e->device);
      st[i] = f(e->groups[i]);
    });
  for (auto& t : th) t.join();
  ch_status r = CH_OK;
  for (ch_status s : st)
    if (s != CH_OK && s != ok_also && r == CH_OK) r = s;
  if (r == CH_OK)
    for (ch_status s : st)
      if (s == ok_also) r = s;
  return r;
}

}  // namespace

extern "C" {

void ch_ensemble_destroy(ch_ensemble* e) {
  if (!e) return;
  for (auto& g : e->groups) {
    ch_parareal_destroy(g.h);
    if (g.st) cudaStreamDestroy(g.st);
  }
  delete e;
}

ch_status ch_ensemble_create(const ch_config* cfg, int nprob, const int* n_per_problem, const double* eps_per_problem,
                             ch_ensemble** out) {
  if (!out) return CH_ERR_INVALID;
  *out = nullptr;
  if (!cfg || cfg->dim != 2 || nprob < 1 || !n_per_problem || !eps_per_problem) return CH_ERR_INVALID;
  ch_ensemble* e = new (std::nothrow) ch_ensemble();
  if (!e) return CH_ERR_OOM;
  e->cfg = *cfg;
  cudaGetDevice(&e->device);
  std::map<int, std::vector<int>> by_n;
  for (int i = 0; i < nprob; ++i) by_n[n_per_problem[i]].push_back(i);
  e->where.assign(nprob, {0, 0});
  for (auto& kv : by_n) {
    ch_ensemble::Group g;
    g.n = kv.first;
    g.problems = kv.second;
    ch_config c = *cfg;
    c.n = g.n;
    c.eps = eps_per_problem[g.problems[0]];
    cudaError_t ce = cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
      ch_ensemble_destroy(e);
      return ce == cudaErrorMemoryAllocation ? CH_ERR_OOM : CH_ERR_CUDA;
    }
    ch_status s = ch_parareal_create(&c, (int)g.problems.size(), g.st, &g.h);
    if (s == CH_OK) {
      std::vector<double> eps(g.problems.size());
      for (size_t j = 0; j < g.problems.size(); ++j) eps[j] = eps_per_problem[g.problems[j]];
      s = ch_parareal_set_eps(g.h, eps.data(), eps.size());
    }
    if (s != CH_OK) {
      if (g.h) ch_parareal_destroy(g.h);
      cudaStreamDestroy(g.st);
      ch_ensemble_destroy(e);
      return s;
    }
    const int gi = (int)e->groups.size();
    for (size_t j = 0; j < g.problems.size(); ++j) e->where[g.problems[j]] = {gi, (int)j};
    e->groups.push_back(g);
  }
  *out = e;
  return CH_OK;
}

const char* ch_ensemble_last_error(const ch_ensemble* e) {
  if (!e) return "NULL handle";
  if (!e->msg.empty()) return e->msg.c_str();
  for (const auto& g : e->groups) {
    const char* m = ch_parareal_last_error(g.h);
    if (m && *m) return m;
  }
  return "";
}

int ch_ensemble_groups(const ch_ensemble* e) { return e ? (int)e->groups.size() : 0; }

ch_status ch_ensemble_set_initial(ch_ensemble* e, int problem, const double* u0_host, size_t len) {
  if (!e) return CH_ERR_INVALID;
  if (problem < 0 || problem >= (int)e->where.size()) return efail(e, CH_ERR_INVALID, "set_initial: bad problem index");
  const auto w = e->where[problem];
  return ch_parareal_set_initial(e->groups[w.first].h, w.second, u0_host, len);
}

ch_status ch_ensemble_compute_reference(ch_ensemble* e) {
  if (!e) return CH_ERR_INVALID;
  return for_groups(e, [](ch_ensemble::Group& g) { return ch_parareal_compute_reference(g.h); }, CH_OK);
}

ch_status ch_ensemble_run(ch_ensemble* e) {
  if (!e) return CH_ERR_INVALID;
  return for_groups(e, [](ch_ensemble::Group& g) { return ch_parareal_run(g.h); }, CH_ERR_NOT_CONVERGED);
}

ch_status ch_ensemble_get_slices(ch_ensemble* e, int problem, double* out_host, size_t len) {
  if (!e) return CH_ERR_INVALID;
  if (problem < 0 || problem >= (int)e->where.size()) return efail(e, CH_ERR_INVALID, "get_slices: bad problem index");
  const auto w = e->where[problem];
  return ch_parareal_get_slices(e->groups[w.first].h, w.second, out_host, len);
}

ch_status ch_ensemble_get_reference(ch_ensemble* e, int problem, double* out_host, size_t len) {
  if (!e) return CH_ERR_INVALID;
  if (problem < 0 || problem >= (int)e->where.size()) return efail(e, CH_ERR_INVALID, "get_reference: bad problem index");
  const auto w = e->where[problem];
  return ch_parareal_get_reference(e->groups[w.first].h, w.second, out_host, len);
}

ch_status ch_ensemble_get_stats(ch_ensemble* e, int problem, ch_stats* out) {
  if (!e) return CH_ERR_INVALID;
  if (problem < 0 || problem >= (int)e->where.size()) return efail(e, CH_ERR_INVALID, "get_stats: bad problem index");
  const auto w = e->where[problem];
  return ch_parareal_get_stats(e->groups[w.first].h, w.second, out);
}

}  // extern "C"
