// Neumann-Neumann fine solver of Section 4.6 (1D), for the linear scheme Eq. 2.4.
//
// A step solves the mixed system of Section 4.6,
//     u - dt D v = u^n,     eps^2 D u - c^2 u + v = -u^n,     c^2 = (u^n)^2 (1 in the frozen model),
// whose elimination of v is Eq. 2.4 exactly (D the three-point Laplacian of Eq. 3.2, u = v = 0 on
// the boundary), over N0 equal subdomains separated by the interface nodes k m - 1 (0-based;
// n + 1 = N0 m). Each interface row of the global system is shared by its two subdomains: the
// terms in u, c^2 u and v half each, the Laplacian split into its one-sided parts, so that the
// local matrices sum to the global one. From the interface values (g, h) = (u^n, v(u^n)), an
// iteration solves the Dirichlet problems (interior rows, interface values fixed), forms the
// residual of the global rows at the interfaces, solves the Neumann problems (local matrix with its
// interface rows, zero data inside, the residual on the interface rows) and adds theta times the
// sum of the two Neumann solutions to each interface value (Richardson iteration on the interface
// Schur complement with the Neumann-Neumann preconditioner); it stops when both updates have
// Euclidean norm over the interfaces <= tol, and the step is the Dirichlet solution for the
// updated interface values. The iteration's fixed point is the global step.
//
// One warp per unit (problem-slice): lane i owns subdomain i and solves its block-tridiagonal
// systems (2x2 blocks (u_j, v_j)) by block elimination in FP64; the unit's state and the
// elimination's intermediates live in shared memory.
#include <cuda_runtime.h>

#include <mutex>
#include <set>

#include "ch_ctx.cuh"
#include "ch1d.cuh"

namespace chg {
namespace {

struct B2 {
  double a, b, c, d;  // [[a, b], [c, d]]
};
struct V2d {
  double x, y;
};

__device__ __forceinline__ B2 mul(const B2& p, const B2& q) {
  return {p.a * q.a + p.b * q.c, p.a * q.b + p.b * q.d, p.c * q.a + p.d * q.c, p.c * q.b + p.d * q.d};
}
__device__ __forceinline__ V2d mul(const B2& p, const V2d& v) { return {p.a * v.x + p.b * v.y, p.c * v.x + p.d * v.y}; }
__device__ __forceinline__ B2 sub(const B2& p, const B2& q) { return {p.a - q.a, p.b - q.b, p.c - q.c, p.d - q.d}; }
__device__ __forceinline__ V2d sub(const V2d& p, const V2d& q) { return {p.x - q.x, p.y - q.y}; }
__device__ __forceinline__ B2 inv(const B2& p) {
  const double r = 1.0 / (p.a * p.d - p.b * p.c);
  return {p.d * r, -p.b * r, -p.c * r, p.a * r};
}

// Coefficients of one unit's step.
struct NNRow {
  double dth;   // dt / h^2
  double e2h;   // eps^2 / h^2
  int frozen;
};

// Diagonal block of node j: the full global row, or the half at an interface end.
__device__ __forceinline__ B2 diag_block(const NNRow& k, double c2, bool half) {
  return half ? B2{0.5, k.dth, -k.e2h - 0.5 * c2, 0.5} : B2{1.0, 2.0 * k.dth, -2.0 * k.e2h - c2, 1.0};
}

// Coupling of a row to a neighbouring node (both directions): u - dt D v, eps^2 D u + v.
__device__ __forceinline__ B2 off_block(const NNRow& k) { return B2{0.0, -k.dth, k.e2h, 0.0}; }

// Block elimination of rows a..b of the subdomain system: diagonal blocks from diag_block (half
// rows where is_half), off-diagonal blocks off_block, right-hand sides rhs(j). tmp: 6 doubles
// per row, private to the caller. Writes the solution to (xu, xv)[a..b] unless xu is null, and
// returns it at rows a and b.
struct Ends {
  V2d first, last;
};

template <typename Rhs, typename Half>
__device__ Ends block_solve(const NNRow& k, const double* un, double* xu, double* xv, double* tmp, int a, int b,
                            Rhs rhs, Half is_half) {
  const B2 L = off_block(k);
  B2 Cp{0.0, 0.0, 0.0, 0.0};
  V2d dp{0.0, 0.0};
  for (int j = a; j <= b; ++j) {
    const double c2 = k.frozen ? 1.0 : un[j] * un[j];
    B2 M = diag_block(k, c2, is_half(j));
    V2d r = rhs(j);
    if (j > a) {
      M = sub(M, mul(L, Cp));
      r = sub(r, mul(L, dp));
    }
    const B2 Mi = inv(M);
    const B2 C = (j < b) ? mul(Mi, L) : B2{0.0, 0.0, 0.0, 0.0};
    const V2d d = mul(Mi, r);
    double* t = tmp + 6 * (j - a);
    t[0] = C.a;
    t[1] = C.b;
    t[2] = C.c;
    t[3] = C.d;
    t[4] = d.x;
    t[5] = d.y;
    Cp = C;
    dp = d;
  }
  V2d x = dp;
  const V2d last = x;
  if (xu) {
    xu[b] = x.x;
    xv[b] = x.y;
  }
  for (int j = b - 1; j >= a; --j) {
    const double* t = tmp + 6 * (j - a);
    const B2 C{t[0], t[1], t[2], t[3]};
    x = sub(V2d{t[4], t[5]}, mul(C, x));
    if (xu) {
      xu[j] = x.x;
      xv[j] = x.y;
    }
  }
  return Ends{x, last};
}

// Shared memory of one warp's unit: the state u^n, the current iterate (u, v) (interior nodes:
// the Dirichlet solutions; interface nodes: the interface values), the interface residuals, the
// Neumann solutions at each subdomain's two ends and the elimination intermediates.
struct NNSmem {
  double* un;   // [n]
  double* xu;   // [n]
  double* xv;   // [n]
  double* ri;   // [2 (N0 - 1)]
  double* wl;   // [2 N0] Neumann solution at the subdomain's left interface
  double* wr;   // [2 N0] ... at its right interface
  double* tmp;  // [N0][m + 1][6]
};

__host__ __device__ inline size_t nn_smem_doubles(int n, int N0) {
  const int m = (n + 1) / N0;
  return (size_t)3 * n + 2 * (N0 - 1) + 4 * N0 + (size_t)N0 * (m + 1) * 6;
}

__device__ inline NNSmem nn_carve(double* base, int n, int N0) {
  const int m = (n + 1) / N0;
  NNSmem s;
  s.un = base;
  s.xu = s.un + n;
  s.xv = s.xu + n;
  s.ri = s.xv + n;
  s.wl = s.ri + 2 * (N0 - 1);
  s.wr = s.wl + 2 * N0;
  s.tmp = s.wr + 2 * N0;
  (void)m;
  return s;
}

// One step of Eq. 2.4 by the Neumann-Neumann iteration, by the calling warp, in place on sm.un.
// Returns the iterations; sets *capped if the cap was reached without convergence.
__device__ int nn_step_warp(const Params1D& p, const NNSmem& sm, bool* capped) {
  const int n = p.n, N0 = p.nn_sub, m = (n + 1) / N0, lane = threadIdx.x & 31;
  const double h2inv = 1.0 / (p.h * p.h);
  const NNRow k{p.dt * h2inv, p.eps2 * h2inv, p.frozen};
  const B2 L = off_block(k);
  const double* un = sm.un;
  // subdomain `lane`: interior nodes lo..hi, interfaces lo - 1 (if lane > 0) and hi + 1 (if
  // lane < N0 - 1)
  const int lo = lane * m, hi = (lane + 1) * m - 2;
  const bool own = lane < N0;
  const bool has_l = own && lane > 0, has_r = own && lane < N0 - 1;
  double* tmp = sm.tmp + (size_t)(own ? lane : 0) * (m + 1) * 6;
  auto c2_of = [&](int j) { return k.frozen ? 1.0 : un[j] * un[j]; };
  // initial interface values: u^n and v from the second equation at u = u^n
  if (has_r) {
    const int g = hi + 1;
    const double lap = (un[g - 1] - 2.0 * un[g] + un[g + 1]) * h2inv;
    sm.xu[g] = un[g];
    sm.xv[g] = -un[g] - p.eps2 * lap + c2_of(g) * un[g];
  }
  __syncwarp();
  auto dirichlet = [&]() {
    if (own)
      block_solve(
          k, un, sm.xu, sm.xv, tmp, lo, hi,
          [&](int j) {
            V2d r{un[j], -un[j]};
            if (j == lo && has_l) r = sub(r, mul(L, V2d{sm.xu[lo - 1], sm.xv[lo - 1]}));
            if (j == hi && has_r) r = sub(r, mul(L, V2d{sm.xu[hi + 1], sm.xv[hi + 1]}));
            return r;
          },
          [](int) { return false; });
    __syncwarp();
  };
  int it = 0;
  bool done = (N0 == 1);
  while (!done) {
    dirichlet();
    // residual of the global rows at the interfaces
    if (has_r) {
      const int g = hi + 1;
      const double u0 = sm.xu[g - 1], u1 = sm.xu[g], u2 = sm.xu[g + 1];
      const double v0 = sm.xv[g - 1], v1 = sm.xv[g], v2 = sm.xv[g + 1];
      sm.ri[2 * lane] = un[g] - (u1 - k.dth * (v0 - 2.0 * v1 + v2));
      sm.ri[2 * lane + 1] = -un[g] - (k.e2h * (u0 - 2.0 * u1 + u2) - c2_of(g) * u1 + v1);
    }
    __syncwarp();
    // Neumann problems: rows a..b including the interface rows, data only on those rows
    if (own) {
      const int a = has_l ? lo - 1 : lo, b = has_r ? hi + 1 : hi;
      const Ends w = block_solve(
          k, un, nullptr, nullptr, tmp, a, b,
          [&](int j) {
            if (has_l && j == a) return V2d{sm.ri[2 * (lane - 1)], sm.ri[2 * (lane - 1) + 1]};
            if (has_r && j == b) return V2d{sm.ri[2 * lane], sm.ri[2 * lane + 1]};
            return V2d{0.0, 0.0};
          },
          [&](int j) { return (has_l && j == a) || (has_r && j == b); });
      sm.wl[2 * lane] = w.first.x;
      sm.wl[2 * lane + 1] = w.first.y;
      sm.wr[2 * lane] = w.last.x;
      sm.wr[2 * lane + 1] = w.last.y;
    }
    __syncwarp();
    // update of the interface values; norms of the updates over the interfaces
    double su = 0.0, sv = 0.0;
    if (has_r) {
      const int g = hi + 1;
      const double du = p.nn_theta * (sm.wr[2 * lane] + sm.wl[2 * (lane + 1)]);
      const double dv = p.nn_theta * (sm.wr[2 * lane + 1] + sm.wl[2 * (lane + 1) + 1]);
      sm.xu[g] += du;
      sm.xv[g] += dv;
      su = du * du;
      sv = dv * dv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      su += __shfl_xor_sync(0xffffffffu, su, o);
      sv += __shfl_xor_sync(0xffffffffu, sv, o);
    }
    ++it;
    const bool conv = sqrt(su) <= p.nn_tol && sqrt(sv) <= p.nn_tol;
    if (!conv && it >= p.nn_max) *capped = true;
    done = conv || it >= p.nn_max;
    __syncwarp();
  }
  // the step: the Dirichlet solution for the final interface values (N0 = 1: the direct solve)
  dirichlet();
  for (int j = lane; j < n; j += 32) sm.un[j] = sm.xu[j];
  __syncwarp();
  return it;
}

// J steps of the unit held in sm.un; NN iterations summed / largest, cap and non-finite flags.
__device__ void nn_propagate_warp(const Params1D& p, const NNSmem& sm, unsigned long long& nsum, int& npeak,
                                  unsigned& status) {
  bool capped = false;
  for (int step = 0; step < p.J; ++step) {
    const int it = nn_step_warp(p, sm, &capped);
    nsum += (unsigned long long)it;
    npeak = it > npeak ? it : npeak;
  }
  bool bad = false;
  for (int j = threadIdx.x; j < p.n; j += 32) bad |= !isfinite(sm.un[j]);
  if (__any_sync(0xffffffffu, bad)) status |= ST_NONFINITE;
  if (capped) status |= ST_NEWTON;
}

// Fine sweep with the NN solver: every active (problem, slice >= k) unit, J steps, F = result.
// One warp per block; blocks take units from the shared counter (persistent grid).
__global__ void __launch_bounds__(32) k_nn_fine_sweep(Params1D p, const double* __restrict__ U, double* __restrict__ F,
                                                      Ctrl* ctrl, ProblemState ps) {
  extern __shared__ double nn_sm[];
  const NNSmem sm = nn_carve(nn_sm, p.n, p.nn_sub);
  __shared__ int unit;
  const int k = ctrl->k;
  const int per = p.N - k;
  if (per <= 0) return;
  const int total = p.B * per;
  for (;;) {
    if (threadIdx.x == 0) unit = atomicAdd(&ctrl->next_unit, 1);
    __syncwarp();
    const int u = unit;
    __syncwarp();
    if (u >= total) break;
    const int b = u / per, s = k + u % per;
    if (!ps.active[b]) continue;
    const double* src = U + ((size_t)b * (p.N + 1) + s) * p.n;
    for (int j = threadIdx.x; j < p.n; j += 32) sm.un[j] = src[j];
    __syncwarp();
    unsigned long long nsum = 0;
    int npeak = 0;
    unsigned status = 0;
    nn_propagate_warp(p, sm, nsum, npeak, status);
    double* dst = F + ((size_t)b * p.N + s) * p.n;
    for (int j = threadIdx.x; j < p.n; j += 32) dst[j] = sm.un[j];
    if (threadIdx.x == 0) {
      atomicAdd(&ps.newton_total[b], nsum);
      atomicMax(&ps.newton_max[b], npeak);
      if (status) atomicOr(&ctrl->status, status);
    }
    __syncwarp();
  }
}

// The sequential fine solution with the NN solver: one warp per problem, Uref[b][s + 1] from
// Uref[b][s] for s = 0..N-1.
__global__ void __launch_bounds__(32) k_nn_reference(Params1D p, double* __restrict__ Uref, Ctrl* ctrl) {
  extern __shared__ double nn_sm[];
  const NNSmem sm = nn_carve(nn_sm, p.n, p.nn_sub);
  const int b = blockIdx.x;
  double* Rb = Uref + (size_t)b * (p.N + 1) * p.n;
  for (int j = threadIdx.x; j < p.n; j += 32) sm.un[j] = Rb[j];
  __syncwarp();
  unsigned long long nsum = 0;
  int npeak = 0;
  unsigned status = 0;
  for (int s = 0; s < p.N; ++s) {
    nn_propagate_warp(p, sm, nsum, npeak, status);
    for (int j = threadIdx.x; j < p.n; j += 32) Rb[(size_t)(s + 1) * p.n + j] = sm.un[j];
    __syncwarp();
  }
  if (threadIdx.x == 0 && status) atomicOr(&ctrl->status, status);
}

// Largest dynamic shared memory of a unit (nn_supported rejects larger sizes).
constexpr size_t kNNMaxSmem = 200 * 1024;

// Opts a kernel into kNNMaxSmem of dynamic shared memory once per device (the attribute is a
// limit: every supported size launches under it).
template <typename K>
cudaError_t nn_prep(K kernel) {
  static std::mutex mu;
  static std::set<std::pair<const void*, unsigned long long>> done;  // (kernel, context)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(reinterpret_cast<const void*>(kernel), chctx::cache_key());
  if (done.count(key)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNNMaxSmem);
  if (e == cudaSuccess) done.insert(key);
  return e;
}

}  // namespace

bool nn_supported(const Params1D& p) {
  return p.nn_sub >= 1 && p.nn_sub <= 32 && (p.n + 1) % p.nn_sub == 0 && (p.n + 1) / p.nn_sub >= 2 &&
         nn_smem_doubles(p.n, p.nn_sub) * sizeof(double) <= kNNMaxSmem;
}

cudaError_t nn_max_grid(const Params1D& p, int* grid) {
  const size_t smem = nn_smem_doubles(p.n, p.nn_sub) * sizeof(double);
  cudaError_t e = nn_prep(k_nn_fine_sweep);
  if (e == cudaSuccess) e = nn_prep(k_nn_reference);
  int dev = 0, sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nn_fine_sweep, 32, smem);
  if (e != cudaSuccess) return e;
  *grid = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

cudaError_t launch_nn_fine_sweep(const Params1D& p, const double* U, double* F, Ctrl* ctrl, ProblemState ps, int grid,
                                 cudaStream_t st) {
  const size_t smem = nn_smem_doubles(p.n, p.nn_sub) * sizeof(double);
  k_nn_fine_sweep<<<grid, 32, smem, st>>>(p, U, F, ctrl, ps);
  return cudaGetLastError();
}

cudaError_t launch_nn_reference(const Params1D& p, double* Uref, Ctrl* ctrl, cudaStream_t st) {
  const size_t smem = nn_smem_doubles(p.n, p.nn_sub) * sizeof(double);
  cudaError_t e = nn_prep(k_nn_reference);
  if (e != cudaSuccess) return e;
  k_nn_reference<<<p.B, 32, smem, st>>>(p, Uref, ctrl);
  return cudaGetLastError();
}

}  // namespace chg
