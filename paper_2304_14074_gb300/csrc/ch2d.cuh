// Two-dimensional Parareal kernels: declarations shared with the host runtime.
#pragma once
#include <cuda_runtime.h>

#include <utility>
#include <vector>

namespace chg2 {

struct PArgs;

enum Scheme { SCHEME_LIN1 = 0, SCHEME_NL = 1, SCHEME_LIN2 = 2 };
enum : unsigned { ST_NEWTON = 1u, ST_NONFINITE = 2u, ST_LINSOLVE = 4u, ST_TIMEOUT = 8u };

// How a batch of implicit steps is executed: one CUDA graph per step (each phase a kernel; the
// Newton and CG loops conditional WHILE nodes, 5 kernels per CG iteration), or one persistent
// cooperative kernel per propagate call (the same phases separated by grid barriers), or plain
// launches with the loops driven from the host (for profiling single kernels), or one
// thread-block cluster per unit running that unit's whole propagation in one launch.
enum StepPath { PATH_GRAPH = 0, PATH_PERSISTENT = 1, PATH_HOST = 2, PATH_CLUSTER = 3 };

// Grid sizes the sine transform supports: n + 1 a power of two in 16..512 (FFTs of length
// 2(n+1), or n + 1 at n = 255 and 511).
bool supported_n(int n);

struct Params2D {
  int n;             // interior nodes per direction
  int frozen;        // diag(u^2) := I (analysis model of Section 3)
  int newton_max;
  int cg_max;        // inner CG iterations per Newton (or refinement) sweep
  double eps2;
  double h;
  double newton_tol;
  double cg_tol;     // relative reduction of the preconditioned residual norm
};

// Work space and kernels of a batch of `cap` units (problem-slices) of an n x n grid.
// All vectors are device arrays [units][n*n], row-major (x fastest).
class Prop2D {
 public:
  cudaError_t init(const Params2D& p, int cap, cudaStream_t st);
  void release();
  // Advances `units` states in place by nsteps steps of `scheme` with step dt. Y: [units][n*n]
  // FP64 device array. Accumulates Newton iterations per unit into newton (device, may be null)
  // and ORs error bits into *status_dev.
  cudaError_t propagate(double* Y, int units, int scheme, double dt, int nsteps, cudaStream_t st);
  cudaError_t propagate_persistent(double* Y, int units, int scheme, double dt, int nsteps, cudaStream_t st);
  cudaError_t propagate_host(double* Y, int units, int scheme, double dt, int nsteps, cudaStream_t st);
  cudaError_t propagate_cluster(double* Y, int units, int scheme, double dt, int nsteps, cudaStream_t st);
  void set_path(StepPath p) { path_ = p; }
  // Per-unit eps^2 (device array [units], row i of the next propagate calls) or null (all units
  // use Params2D::eps2). Graphs built afterwards read the array at every replay.
  void set_unit_eps2(const double* eps2_dev) {
    if (eps2_dev != eps2u_) {
      for (auto& c : graphs_) cudaGraphExecDestroy(c.second);
      graphs_.clear();
    }
    eps2u_ = eps2_dev;
  }
  StepPath path() const { return path_; }
  int cluster_size() const { return cluster_size_; }
  // Orthonormal 2D DST-I (its own inverse) of `units` FP32 fields; in and out must differ and
  // must not be the internal scratch buffers.
  cudaError_t dst2(const float* in, float* out, int units, cudaStream_t st);
  unsigned read_status(cudaStream_t st);  // synchronises
  // Clears status bits (enqueued on st): a failure the caller has handled (a learned coarse
  // prediction that the guard replaces) is not reported at the end of the run.
  cudaError_t clear_status(unsigned mask, cudaStream_t st);
  unsigned long long newton_iterations() const { return newton_total_; }
  long long cg_iterations() const { return cg_total_; }
  long long cg_unit_iterations() const { return cg_unit_total_; }  // summed over units
  int newton_peak() const { return newton_peak_; }
  // Kernels launched by the step graphs since the last reset (as of the last read_status): each
  // step runs a fixed prologue and epilogue, each batched Newton pass kNewtonKernels and each
  // batched CG iteration kCgKernels.
  long long kernel_launches() const {
    if (path_ == PATH_PERSISTENT || path_ == PATH_CLUSTER) return step_kernels_;
    if (path_ == PATH_HOST) return step_kernels_ + (kNewtonKernels - 2) * newton_passes_ + kCgKernels * cg_total_;
    return step_kernels_ + kNewtonKernels * newton_passes_ + kCgKernels * cg_total_;
  }
  static constexpr int kStepKernelsNL = 3;   // prologue, predictor, loop start
  static constexpr int kStepKernelsLin = 3;
  static constexpr int kNewtonKernels = 9;   // z, residual, 2 transform passes (the second starts CG),
                                             // CG loop start, 2 passes (last CG update, Newton
                                             // update), stop test, condition
  static constexpr int kCgKernels = 5;       // 4 transform passes (the first applies the previous
                                             // iteration's update), scalars and condition
  // Zeroes the device status bits and the Newton / CG counters (enqueued on st).
  cudaError_t reset_counters(cudaStream_t st);
  size_t bytes() const { return bytes_; }

 private:
  struct StepKey {
    double* Y;
    int units;
    int scheme;
    double dt;
    int have_prev;
    int u0;     // first unit of the group (offset into the work arrays)
    int group;  // loop-control slots of the group
    bool operator==(const StepKey& o) const {
      return Y == o.Y && units == o.units && scheme == o.scheme && dt == o.dt && have_prev == o.have_prev &&
             u0 == o.u0 && group == o.group;
    }
  };
  static constexpr int kMaxGroups = 4;       // concurrent unit groups of a propagation
  static constexpr int kMinGroupUnits = 8;   // units per group at least
  cudaError_t build_step(const StepKey& k, cudaGraphExec_t* out);
  void make_args(PArgs& a, double* Y, int units, int scheme, double dt, int nsteps, int u0, int group) const;
  cudaStream_t gs_[4] = {};   // group streams
  cudaEvent_t gev_[4] = {};   // group joins
  cudaEvent_t gfork_ = nullptr;
  std::vector<std::pair<StepKey, cudaGraphExec_t>> graphs_;

  Params2D p_{};
  int cap_ = 0;
  size_t pts_ = 0;
  size_t bytes_ = 0;
  int nblk_ = 0;  // reduction blocks per unit
  // FP64 work
  double* yhat_ = nullptr;   // (I - dt D_h) u^n, or the linear right-hand side
  double* yprev_ = nullptr;  // u^{n-1} for the Newton predictor
  double* z_ = nullptr;      // stencil intermediate
  double* xacc_ = nullptr;   // accumulated solution of a refined linear solve
  // FP32 work
  float* w_ = nullptr;       // Jacobian weights (Y^2 or u^2)
  float* rhs_ = nullptr;     // right-hand side handed to CG
  float* xh_ = nullptr;      // CG iterate (spectral)
  float* rh_ = nullptr;      // CG residual (spectral)
  float* ph_ = nullptr;      // CG direction (spectral)
  float* qh_ = nullptr;      // S p (spectral)
  float* tmp_ = nullptr;     // transform scratch / physical-space work
  float* tmp2_ = nullptr;
  float* mu_ = nullptr;      // 1D eigenvalues mu_p of -D_h, p = 1..n
  float2* tw_ = nullptr;     // FFT twiddles exp(-2 pi i m / L), m < L
  // per-unit scalars
  double* part_ = nullptr;   // reduction partials [units][nblk]
  double* scal_ = nullptr;   // [units][8]: rho, rho0, alpha, beta, wbar, dmax, prevd, spare
  int* flag_ = nullptr;      // [units][2]: newton done, cg done
  int* newton_cnt_ = nullptr;  // [units] Newton iterations of the current step
  unsigned* status_ = nullptr;
  int* ctr_ = nullptr;         // per group: [0] Newton, [1] CG iteration; [2], [3] the CG scalar kernel's sum and arrivals
  unsigned long long* cg_dev_ = nullptr;  // CG iterations (batched) since the last reset
  int* host_cnt_ = nullptr;    // pinned
  unsigned long long newton_total_ = 0;
  int newton_peak_ = 0;
  long long cg_total_ = 0;
  long long newton_passes_ = 0;
  long long cg_unit_total_ = 0;
  long long step_kernels_ = 0;
  StepPath path_ = PATH_GRAPH;
  const double* eps2u_ = nullptr;  // per-unit eps^2 or null
  int persist_minb_ = 3;
  int cluster_force_ = 0;     // cluster execution: cluster size (0: chosen by residency)
  int cluster_size_ = 0;      // cluster size of the last cluster launch      // persistent path: blocks per SM it is compiled for (2, 3, 4)
  double* ppart_ = nullptr;   // persistent path: per-item partial sums [7][cap][rows / 16]
  int* active_ = nullptr;     // persistent path: units still iterating (parity slots)
  unsigned* bar_ = nullptr;   // persistent path: grid barrier (arrivals, generation, abort)
  double* cgs_ = nullptr;     // CG scalars per unit
  float* uh_ = nullptr;       // CG u = M^{-1} r (sine space)
  float* sh_ = nullptr;       // CG s = S p (sine space)
};

// Parareal correction of one slice for `count` problems list[0..count) (Eq. 2.2), fused with
// the increment and error norms: U_{s+1} = F_s + (g - Gold_s) (init: U_{s+1} = g), Gold_s = g,
// and g (work rows, contiguous) is overwritten with U_{s+1}. U, F, Gold point at slice s+1 / s
// of problem 0; ustride / fstride are the per-problem strides. acc[b] = {inc, err_l2, err_max,
// max |U_{s+1}| (infinite if not finite)} are running maxima over slices (h2 = h^d for the L2_h
// norm). part: correct_partials(count).
cudaError_t launch_correct(double* U, const double* F, double* g, double* Gold, const double* Uref, const int* list,
                           int count, size_t pts, size_t ustride, size_t fstride, int init, double* part, double* acc,
                           double h2, cudaStream_t st);
size_t correct_partials(int count);
// dst[i] = src[off[i] .. off[i] + pts) (gather) and the converse (scatter).
cudaError_t launch_gather(double* dst, const double* src, const long long* off, int count, size_t pts, cudaStream_t st);
cudaError_t launch_scatter(double* dst, const double* src, const long long* off, int count, size_t pts,
                           cudaStream_t st);

}  // namespace chg2
