// Learned coarse propagator G_theta(U) = U + R(U): declarations shared with the host runtime.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

namespace chg3 {

constexpr int kC = 32;  // hidden channels
// Flat parameter layout (FP32): for each layer l = 0..5, W_l [3][3][Cout][Cin] then b_l [Cout];
// channels 1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1.
constexpr int kOffW[6] = {0, 320, 9568, 18816, 28064, 37312};
constexpr int kOffB[6] = {288, 9536, 18784, 28032, 37280, 37600};
constexpr int kParams = 37601;
constexpr int kTrainMargin = 6;  // receptive-field radius of six 3 x 3 layers
inline int train_crop(int n) { return n + 2 * kTrainMargin < 76 ? n + 2 * kTrainMargin : 76; }

class GTheta {
 public:
  static constexpr int kForwardKernels = 6;  // launches of one forward64
  cudaError_t init(unsigned long long seed, cudaStream_t st);
  void release();
  cudaError_t set_params(const float* host, cudaStream_t st);
  cudaError_t get_params(float* host, cudaStream_t st);
  // out = base + R(in) for `batch` FP64 fields of size S x S (base = in when null; out may alias
  // in or base).
  cudaError_t forward64(const double* in, const double* base, double* out, int batch, int S, cudaStream_t st);
  // One forward / backward on FP32 crops (size S, loss on the window [margin, S - margin)^2);
  // leaves the gradients in grad_ and the loss in loss_dev_[slot].
  cudaError_t grad_step(const float* in, const float* target, int batch, int S, int margin, int slot,
                        cudaStream_t st);
  // Adam over `steps` minibatches of random crops of pairs (states[t][s], states[t][s + stride]),
  // fitting R(states[t][s]) to states[t][s + stride] - base[t][s] (base = states when null);
  // states, base: FP64 [ntraj][nsnap][n][n].
  cudaError_t train(const double* states, const double* base, int ntraj, int nsnap, int n, int stride, int steps, int batch,
                    double lr, unsigned long long seed, cudaStream_t st);
  cudaError_t read_losses(float* host, int count, cudaStream_t st);
  // The forward pass of `batch` FP64 fields, keeping every layer's output: out (device, FP32)
  // receives a1..a5 as [5][batch][S][S][32] (the stored BF16 values) followed by R [batch][S][S].
  cudaError_t activations(const double* in, int batch, int S, float* out, cudaStream_t st);
  const float* grads() const { return grad_; }
  // Loss of grad_step / train: false = mean squared error on the windows; true = each crop's
  // squared error over its target's energy on the window, averaged over the batch.
  void set_relative_loss(bool on) { rel_loss_ = on; }
  // 1 if a bounded wait of the tcgen05 path gave up since the handle was created (synchronises).
  int wait_failures(cudaStream_t st);

 private:
  cudaError_t ensure(int batch, int S);
  cudaError_t ensure_losses(int count, cudaStream_t st);
  cudaError_t refresh_bf16(cudaStream_t st);
  cudaError_t forward_acts(const void* in, bool in64, int batch, int S, cudaStream_t st);
  void reduce_tiles(int tiles, int stride, int len, int dst_w, int wlen, int dst_b, cudaStream_t st);

  float* master_ = nullptr;  // kParams
  float* grad_ = nullptr;
  float* m_ = nullptr;
  float* v_ = nullptr;
  __nv_bfloat16* wmid_ = nullptr;   // [4][9][32][32] forward weights of the 32 -> 32 layers
  __nv_bfloat16* wbwd_ = nullptr;   // [4][9][32][32] flipped taps, swapped channels (backward data)
  float* loss_dev_ = nullptr;       // per-step loss history
  int loss_cap_ = 0;
  int adam_t_ = 0;
  // activation workspace
  int cap_batch_ = 0, cap_S_ = 0;
  float* a0_ = nullptr;             // [B][S][S] input (FP32)
  __nv_bfloat16* act_[5] = {};      // a1..a5 [B][S][S][32]
  float* r_ = nullptr;              // [B][S][S] R(U)
  float* dr_ = nullptr;             // [B][S][S] dLoss/dR
  __nv_bfloat16* g_[2] = {};        // gradient ping-pong [B][S][S][32]
  float* part_ = nullptr;           // weight-gradient partials [tiles][len]
  double* part2_ = nullptr;         // their sums over chunks of tiles
  size_t part_cap_ = 0;
  float* tgt_ = nullptr;            // [B][S][S] crop targets
  int4* crops_ = nullptr;           // crop descriptors
  double* lpart_ = nullptr;         // loss partials
  double* eng_ = nullptr;           // [B] target energy of each crop (relative loss)
  bool rel_loss_ = false;
  int* err_ = nullptr;              // a bounded tensor-core wait gave up (tcgen05 path)
  bool tc_ = false;                 // 32 -> 32 layers on tcgen05.mma instead of mma.sync
};

}  // namespace chg3
