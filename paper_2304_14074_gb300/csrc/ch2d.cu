// Two-dimensional fine and coarse propagators for the Cahn-Hilliard Parareal (sm_103a).
//
// Grid: n x n interior nodes of (0,1)^2, h = 1/(n+1), row-major, zero boundary values;
// D_h = I (x) D_1 + D_1 (x) I, the natural extension of Eq. 3.2 (remark closing Section 3).
// A batch of `units` states (problem-slices) is advanced together.
//
// Each implicit step is an FP64 Newton iteration on the step residual H(X) = 0:
//   nonlinear scheme Eq. 2.3 (Eq. 3.17): H(Y) = Y - Yhat + D_h z,  z = eps^2 dt D_h Y - dt Y^3;
//   linear schemes Eq. 2.4 / 2.5:      H(X) = J X - b (one or two sweeps: iterative refinement).
// The correction solves J d = H with J = I + eps^2 dt A^2 + dt A diag(wc), A = -D_h (wc = 3Y^2
// for Eq. 2.3, (u^n)^2 for Eq. 2.4, 2 for Eq. 2.5). J is not symmetric, but A^{-1} J =
// A^{-1} + eps^2 dt A + dt diag(wc) =: S is symmetric positive definite, so we run
// preconditioned CG on S d = A^{-1} H. Split S = M + dt (diag(wc) - wbar I) with
// M = A^{-1} + eps^2 dt A + dt wbar I, which the orthonormal 2D sine transform (DST-I)
// diagonalises: m(p,q) = 1/mu + eps^2 dt mu + dt wbar, mu = mu_p + mu_q the eigenvalues of A.
// The whole CG therefore lives in sine space: each iteration is one inverse transform of the
// direction, one pointwise product with dt (wc - wbar), one forward transform, and diagonal
// updates. No stencil is applied in FP32: the stiff part (entries ~ eps^2 dt / h^4) is exact
// on the diagonal, so FP32 CG reaches ~1e-6 relative accuracy; the FP64 residual sets the
// attainable accuracy of each step.
//
// DST-I: the sine transform of length n is computed from a complex FFT, two real rows packed as
// the real and imaginary parts of one complex FFT: up to n = 127 of length L = 2(n+1), the odd
// extension of the rows (mixed radix-8 Stockham, butterflies in registers, one shared memory
// buffer; the first stage reads the rows from global memory); at n = 255 and 511 of length n + 1
// (fft_rows_half: warp four-step FFTs and a running sum). Each pass transforms rows and writes
// them transposed, so two passes give S X S (S the orthonormal DST-I matrix, S^2 = I).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "ch_ctx.cuh"
#include "ch2d.cuh"

namespace chg2 {

bool supported_n(int n) {
  const int N = n + 1;
  return N == 16 || N == 32 || N == 64 || N == 128 || N == 256 || N == 512;
}

namespace {

constexpr int kDstRows = 16;  // rows per CTA in a transform pass (8 complex FFTs)
constexpr int kBlk = 32;      // CTAs per unit in pointwise kernels (fixed: deterministic reductions)
constexpr int kThreads = 256;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Radix-R DFT in registers, R in {2, 4, 8}: V_s = sum_r v_r exp(-2 pi i r s / R).
template <int R>
__device__ __forceinline__ void dft_small(float2 (&v)[R]);
template <>
__device__ __forceinline__ void dft_small<2>(float2 (&v)[2]) {
  const float2 a = v[0], b = v[1];
  v[0] = make_float2(a.x + b.x, a.y + b.y);
  v[1] = make_float2(a.x - b.x, a.y - b.y);
}
template <>
__device__ __forceinline__ void dft_small<4>(float2 (&v)[4]) {
  const float2 a0 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
  const float2 a1 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
  const float2 a2 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
  const float2 a3 = make_float2(v[1].y - v[3].y, v[3].x - v[1].x);  // -i (v1 - v3)
  v[0] = make_float2(a0.x + a2.x, a0.y + a2.y);
  v[2] = make_float2(a0.x - a2.x, a0.y - a2.y);
  v[1] = make_float2(a1.x + a3.x, a1.y + a3.y);
  v[3] = make_float2(a1.x - a3.x, a1.y - a3.y);
}
template <>
__device__ __forceinline__ void dft_small<8>(float2 (&v)[8]) {
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft_small<4>(e);
  dft_small<4>(o);
  const float r2 = 0.70710678118654752f;
  // o_s *= W8^s, W8 = exp(-2 pi i / 8)
  const float2 o1 = make_float2((o[1].x + o[1].y) * r2, (o[1].y - o[1].x) * r2);
  const float2 o2 = make_float2(o[2].y, -o[2].x);
  const float2 o3 = make_float2((o[3].y - o[3].x) * r2, -(o[3].x + o[3].y) * r2);
  v[0] = make_float2(e[0].x + o[0].x, e[0].y + o[0].y);
  v[4] = make_float2(e[0].x - o[0].x, e[0].y - o[0].y);
  v[1] = make_float2(e[1].x + o1.x, e[1].y + o1.y);
  v[5] = make_float2(e[1].x - o1.x, e[1].y - o1.y);
  v[2] = make_float2(e[2].x + o2.x, e[2].y + o2.y);
  v[6] = make_float2(e[2].x - o2.x, e[2].y - o2.y);
  v[3] = make_float2(e[3].x + o3.x, e[3].y + o3.y);
  v[7] = make_float2(e[3].x - o3.x, e[3].y - o3.y);
}

// Odd extension of a row pair: y_m = (x0[m-1], x1[m-1]) for 0 < m < N, 0 at m = 0 and m = N,
// y_{L-m} = -y_m. r0, r1 are valid rows; v0, v1 = false stands for a zero row past the grid.
// The loads are unconditional (from a valid element), so all of a thread's loads of a stage
// are in flight together; the zeros are selected afterwards.
template <int N>
__device__ __forceinline__ float2 odd_ext(const float* __restrict__ r0, const float* __restrict__ r1, bool v0,
                                          bool v1, int m) {
  constexpr int L = 2 * N;
  const bool zero = (m == 0 || m == N), neg = m > N;
  const int q = zero ? 0 : (neg ? L - m - 1 : m - 1);
  const float a = __ldcg(r0 + q), b = __ldcg(r1 + q);
  const float sa = (zero || !v0) ? 0.f : (neg ? -a : a);
  const float sb = (zero || !v1) ? 0.f : (neg ? -b : b);
  return make_float2(sa, sb);
}

// Shared-memory index with one padding element every 8 complex values: the radix-8 stores of
// the early stages write with strides of 8 and 64 elements, which would otherwise hit the same
// banks (16-way conflicts at stride 8).
__host__ __device__ constexpr int pad8(int x) { return x + (x >> 3); }

// Length of the complex FFT behind a DST-I of length N - 1: 2N (odd extension, two rows packed)
// except on the 256 x 256 and 512 x 512 grids, whose rows are transformed through an FFT of
// length N (fft_rows_half).
template <int N>
__host__ __device__ constexpr int fft_len() {
  return (N == 512 || N == 256) ? N : 2 * N;
}

// Row stride (complex values) of the transform buffer: a padded row of the FFT length L plus one
// value, so that the eight row pairs an epilogue half-warp reads start in eight different banks
// (a stride of 9L/8 complex values is a multiple of 32 words: all eight in one bank).
template <int N>
__host__ __device__ constexpr int buf_row() {
  return fft_len<N>() + fft_len<N>() / 8 + 1;
}
template <int N>
__host__ __device__ constexpr int buf_elems() {
  return (kDstRows / 2) * buf_row<N>();
}

// One Stockham stage of radix R on the F complex FFTs of length L held in buf (in place: all
// items are loaded to registers, then the block synchronises, then results are stored).
// Stage 0 (Ns = 1, all twiddles 1) reads the odd extension of the input rows straight from
// global memory. The twiddles of a later stage are tws[(r - 1) Ns + k] = exp(-2 pi i r k /
// (R Ns)), r = 1..R-1, k < Ns: the threads of a warp read consecutive k (no bank conflicts).
template <int N, int R, int F, bool FIRST>
__device__ __forceinline__ void fft_stage(float2* buf, const float2* tws, int Ns, const float* src, int a0) {
  constexpr int L = 2 * N, LR = L / R, ITEMS = F * LR;
  constexpr int IPT = (ITEMS + kThreads - 1) / kThreads;
  constexpr int n = N - 1;
  float2 v[IPT][R];
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int it = threadIdx.x + q * kThreads;
    if (it < ITEMS) {
      const int f = it / LR, j = it - f * LR;
      if (FIRST) {
        const int ra = a0 + 2 * f, rb = ra + 1;
        const float* r0 = src + (size_t)(ra < n ? ra : 0) * n;
        const float* r1 = src + (size_t)(rb < n ? rb : 0) * n;
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = odd_ext<N>(r0, r1, ra < n, rb < n, j + r * LR);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = buf[f * buf_row<N>() + pad8(j + r * LR)];
      }
    }
  }
  if (!FIRST) __syncthreads();
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int it = threadIdx.x + q * kThreads;
    if (it < ITEMS) {
      const int f = it / LR, j = it - f * LR;
      const int k = FIRST ? 0 : (j & (Ns - 1));
      if (!FIRST) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], tws[(r - 1) * Ns + k]);
      }
      dft_small<R>(v[q]);
      const int o = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[f * buf_row<N>() + pad8(o + r * Ns)] = v[q][r];
    }
  }
  __syncthreads();
}

// Complex FFT of length L = 2N of F rows: radix-8 stages, then one radix-2 or radix-4 stage.
// twd: the per-stage twiddle tables of the stages after the first, one after the other
// (twiddle_table below).
template <int N, int F>
__device__ __forceinline__ void fft_rows(float2* buf, const float2* twd, const float* src, int a0) {
  constexpr int L = 2 * N;
  constexpr int lg = (L == 32) ? 5 : (L == 64) ? 6 : (L == 128) ? 7 : (L == 256) ? 8 : (L == 512) ? 9 : 10;
  constexpr int n8 = lg / 3, rem = lg - 3 * n8;
  static_assert(n8 >= 1, "transform length too short");
  fft_stage<N, 8, F, true>(buf, twd, 1, src, a0);
  int Ns = 8, off = 0;
#pragma unroll
  for (int s = 1; s < n8; ++s) {
    fft_stage<N, 8, F, false>(buf, twd + off, Ns, nullptr, 0);
    off += 7 * Ns;
    Ns *= 8;
  }
  if constexpr (rem == 1) fft_stage<N, 2, F, false>(buf, twd + off, Ns, nullptr, 0);
  if constexpr (rem == 2) fft_stage<N, 4, F, false>(buf, twd + off, Ns, nullptr, 0);
}

// ---- Warp FFTs (the 256 x 256 and 512 x 512 grids). The Stockham version above makes a pass
// through shared memory with a block barrier per stage; here each row pair's FFT is done by one
// warp as a Cooley-Tukey four-step FFT (an FFT over m1 in registers, the twiddles, a transpose
// through the warp's own buffer row, FFTs over t split across lane groups), with one shared-
// memory round trip and warp barriers only; the result is stored where the Stockham version
// leaves it, so the pass epilogues read it unchanged.

// exp(-2 pi i j / 32), j < 16: cos and sin of the angle, rounded to FP32 (host libm values).
__device__ __forceinline__ float2 w32(int j) {
  switch (j) {
    case 1: return make_float2(9.807852804e-01f, -1.950903220e-01f);
    case 2: return make_float2(9.238795325e-01f, -3.826834324e-01f);
    case 3: return make_float2(8.314696123e-01f, -5.555702330e-01f);
    case 4: return make_float2(7.071067812e-01f, -7.071067812e-01f);
    case 5: return make_float2(5.555702330e-01f, -8.314696123e-01f);
    case 6: return make_float2(3.826834324e-01f, -9.238795325e-01f);
    case 7: return make_float2(1.950903220e-01f, -9.807852804e-01f);
    case 9: return make_float2(-1.950903220e-01f, -9.807852804e-01f);
    case 10: return make_float2(-3.826834324e-01f, -9.238795325e-01f);
    case 11: return make_float2(-5.555702330e-01f, -8.314696123e-01f);
    case 12: return make_float2(-7.071067812e-01f, -7.071067812e-01f);
    case 13: return make_float2(-8.314696123e-01f, -5.555702330e-01f);
    case 14: return make_float2(-9.238795325e-01f, -3.826834324e-01f);
    case 15: return make_float2(-9.807852804e-01f, -1.950903220e-01f);
    default: return make_float2(1.f, 0.f);
  }
}

// a W_32^j (j known at compile time after unrolling: 1 and -i multiply by nothing).
__device__ __forceinline__ float2 twmul32(float2 a, int j) {
  if (j == 0) return a;
  if (j == 8) return make_float2(a.y, -a.x);
  return cmul(a, w32(j));
}

// 8- or 16-point FFT in registers, radix-2 decimation in frequency: on return v[i] =
// X[bitrev3(i)] or X[bitrev4(i)]. The stage twiddle W_(2 span)^j is W_32^(j 16 / span).
template <int L>
__device__ __forceinline__ void fft_dif(float2 (&v)[L]) {
  static_assert(L == 8 || L == 16, "register FFT length");
#pragma unroll
  for (int span = L / 2; span >= 1; span >>= 1) {
#pragma unroll
    for (int start = 0; start < L; start += 2 * span) {
#pragma unroll
      for (int j = 0; j < span; ++j) {
        const float2 a = v[start + j], b = v[start + j + span];
        v[start + j] = make_float2(a.x + b.x, a.y + b.y);
        v[start + j + span] = twmul32(make_float2(a.x - b.x, a.y - b.y), j * (16 / span));
      }
    }
  }
}

__host__ __device__ constexpr int bitrev3(int i) { return ((i & 1) << 2) | (i & 2) | ((i & 4) >> 2); }
__host__ __device__ constexpr int bitrev4(int i) {
  return ((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3);
}

// A 512-point FFT of one row pair by one warp, 16 values per lane (four-step, 512 = 32 x 16): on
// entry lane t holds v[m1] = y[32 m1 + t], m1 < 16; a 16-point FFT over m1 in registers; the
// twiddles W_512^(t k1) (table tw2[k1][t]); a transpose through the warp's buffer row s (rows
// padded to 34 entries: the lane pairs below then read distinct banks); then each 32-point FFT
// over t, for one k1, is split across the lane pair (2 k1, 2 k1 + 1): each lane a 16-point FFT of
// the even / odd samples (E, O), and one shuffle combines them, X[k1 + 16 k2] = E[k2] +
// W_32^k2 O[k2] (even lane, k2 < 16) and X[k1 + 16 (k2 + 16)] = E[k2] - W_32^k2 O[k2] (odd lane).
// On return X[k] is at s[pad8(k)], k < 512.
__device__ __forceinline__ void fft512_warp(float2 (&v)[16], float2* s, const float2* tw2, int t) {
  fft_dif<16>(v);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int k1 = bitrev4(i);
    s[k1 * 34 + t] = cmul(v[i], tw2[k1 * 32 + t]);
  }
  __syncwarp();
  const int k1 = t >> 1, odd = t & 1;
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = s[k1 * 34 + 2 * m + odd];
  __syncwarp();
  fft_dif<16>(v);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int k2 = bitrev4(i);
    const float2 w = odd ? twmul32(v[i], k2) : v[i];  // odd lane: W_32^k2 O
    const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, w.x, 1), __shfl_xor_sync(0xffffffffu, w.y, 1));
    const float2 X = odd ? make_float2(o.x - w.x, o.y - w.y) : make_float2(w.x + o.x, w.y + o.y);
    s[pad8(k1 + 16 * (k2 + 16 * odd))] = X;
  }
}

// A 256-point FFT of one row pair by one warp, 8 values per lane (four-step, 256 = 8 x 32): on
// entry lane t holds v[m1] = y[32 m1 + t], m1 < 8; an 8-point FFT over m1 in registers; the
// twiddles W_256^(t k1) (table tw2[k1][t]); a transpose through the warp's buffer row s (rows
// padded to 36 entries: a half-warp's reads below then fall in distinct banks); then the 32-point
// FFT over t for one k1 is split across the lane quad 4 k1 + q: lane q takes the samples
// t = 4 m + q, an 8-point FFT E_q over m, and two shuffle steps combine the quad: with
// q = q0 + 2 q1, G_q0[k' + 8 q1] = E_q0[k'] +- W_16^k' E_(q0+2)[k'] (partners 2 apart), then
// X[k'' + 16 q0] = G_0[k''] +- W_32^k'' G_1[k''] (partners 1 apart), k'' = k' + 8 q1. On return
// X[k] is at s[pad8(k)], k < 256.
__device__ __forceinline__ void fft256_warp(float2 (&v)[8], float2* s, const float2* tw2, int t) {
  constexpr int R = 36;
  fft_dif<8>(v);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k1 = bitrev3(i);
    s[k1 * R + t] = cmul(v[i], tw2[k1 * 32 + t]);
  }
  __syncwarp();
  const int k1 = t >> 2, q0 = t & 1, q1 = (t >> 1) & 1;
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = s[k1 * R + 4 * m + (t & 3)];
  __syncwarp();
  fft_dif<8>(v);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int kp = bitrev3(i);
    // partners 2 apart: the q1 = 1 lane holds E_(q0+2), scaled by W_16^kp = W_32^(2 kp)
    float2 w = q1 ? twmul32(v[i], 2 * kp) : v[i];
    float2 o = make_float2(__shfl_xor_sync(0xffffffffu, w.x, 2), __shfl_xor_sync(0xffffffffu, w.y, 2));
    const float2 g = q1 ? make_float2(o.x - w.x, o.y - w.y) : make_float2(w.x + o.x, w.y + o.y);
    // partners 1 apart: the q0 = 1 lane holds G_1[k''], scaled by W_32^k'' = W_32^kp (-i)^q1
    float2 gt = twmul32(g, kp);
    if (q1) gt = make_float2(gt.y, -gt.x);
    w = q0 ? gt : g;
    o = make_float2(__shfl_xor_sync(0xffffffffu, w.x, 1), __shfl_xor_sync(0xffffffffu, w.y, 1));
    const float2 X = q0 ? make_float2(o.x - w.x, o.y - w.y) : make_float2(w.x + o.x, w.y + o.y);
    s[pad8(k1 + 8 * (kp + 8 * q1 + 16 * q0))] = X;
  }
}

// The 256 x 256 and 512 x 512 grids: the DST-I of length N - 1 of each row from an FFT of length
// N (half the odd extension's), one warp per row pair. With y_0 = y_N = 0 and s_j = sin(pi j / N),
//   w_j = s_j (y_j + y_{N-j}) + (y_j - y_{N-j}) / 2,   j < N,
// and W = FFT(w) (W_k = sum_j w_j e^{-2 pi i j k / N}), the sine coefficients
// F_m = sum_j y_j sin(pi j m / N) are F_{2k} = -Im W_k and F_{2k+1} = F_{2k-1} + Re W_k
// (F_1 = Re W_0 / 2): the symmetric part of w carries the odd coefficients as differences, the
// antisymmetric part the even ones (Numerical Recipes' sine transform, written here from that
// identity). The two rows are packed as z = w_a + i w_b; W_a, W_b are split from Z_k and
// conj(Z_{N-k}), and the odd coefficients summed by a warp scan (each lane N / 64 consecutive k).
// The buffer row then holds what the odd-extension FFT of length 2N would have produced,
// (2 F_m(b), -2 F_m(a)) at pad8(m), so the pass epilogues are the same for every grid.
// twd: tw2[N / 32][32] of the warp FFT, then s_j, j < N, as floats.
template <int N>
__device__ __forceinline__ void fft_rows_half(float2* buf, const float2* twd, const float* src, int a0) {
  static_assert((N == 512 || N == 256) && kDstRows == 16 && kThreads == 256, "one warp per row pair");
  constexpr int n = N - 1, VPL = N / 32, KPL = N / 64;
  static_assert(pad8(N - 1) < buf_row<N>() && (N == 512 ? 16 * 34 : 7 * 36 + 32) <= buf_row<N>(),
                "the FFT fits the buffer row");
  const int f = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int ra = a0 + 2 * f, rb = ra + 1;
  const bool va = ra < n, vb = rb < n;
  const float* r0 = src + (size_t)(va ? ra : 0) * n;
  const float* r1 = src + (size_t)(vb ? rb : 0) * n;
  const float* sj = reinterpret_cast<const float*>(twd + N);
  float2* s = buf + f * buf_row<N>();
  float2 v[VPL];
#pragma unroll
  for (int m1 = 0; m1 < VPL; ++m1) {
    const int j = 32 * m1 + t;
    const bool in = j > 0;  // y_0 = y_N = 0
    const int q = in ? j - 1 : 0, qr = in ? N - j - 1 : 0;
    const float a = __ldcg(r0 + q), ar = __ldcg(r0 + qr), b = __ldcg(r1 + q), br = __ldcg(r1 + qr);
    const float sn = sj[j];
    const float wa = fmaf(sn, a + ar, 0.5f * (a - ar)), wb = fmaf(sn, b + br, 0.5f * (b - br));
    v[m1] = make_float2((in && va) ? wa : 0.f, (in && vb) ? wb : 0.f);
  }
  if constexpr (N == 512) {
    fft512_warp(v, s, twd, t);
  } else {
    fft256_warp(v, s, twd, t);
  }
  __syncwarp();
  // Lane t: k = KPL t + i. W_a = (Z_k + conj Z_{N-k}) / 2, W_b = (Z_k - conj Z_{N-k}) / (2i).
  float ea[KPL], eb[KPL], oa[KPL], ob[KPL];
  float sa = 0.f, sb = 0.f;
#pragma unroll
  for (int i = 0; i < KPL; ++i) {
    const int k = KPL * t + i;
    const float2 z = s[pad8(k)], zr = s[pad8((N - k) & (N - 1))];
    const float war = 0.5f * (z.x + zr.x), wai = 0.5f * (z.y - zr.y);
    const float wbr = 0.5f * (z.y + zr.y), wbi = -0.5f * (z.x - zr.x);
    ea[i] = -wai;  // F_{2k} (row a); unused at k = 0
    eb[i] = -wbi;
    sa += (k == 0) ? 0.5f * war : war;  // running sums: F_{2k+1} of this lane's part
    sb += (k == 0) ? 0.5f * wbr : wbr;
    oa[i] = sa;
    ob[i] = sb;
  }
  // exclusive warp scan of the lanes' totals
  float pa = sa, pb = sb;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float qa = __shfl_up_sync(0xffffffffu, pa, o), qb = __shfl_up_sync(0xffffffffu, pb, o);
    if (t >= o) {
      pa += qa;
      pb += qb;
    }
  }
  pa -= sa;
  pb -= sb;
  __syncwarp();  // every lane has read Z before any lane overwrites it
#pragma unroll
  for (int i = 0; i < KPL; ++i) {
    const int k = KPL * t + i;
    if (k > 0) s[pad8(2 * k)] = make_float2(2.f * eb[i], -2.f * ea[i]);
    s[pad8(2 * k + 1)] = make_float2(2.f * (pb + ob[i]), -2.f * (pa + oa[i]));
  }
}

// The row FFTs of a transform pass (the warp versions at 512 x 512 and 256 x 256); ends with a
// block barrier, after which `buf` holds the transforms for the epilogue.
template <int N, int F>
__device__ __forceinline__ void fft_rows_any(float2* buf, const float2* twd, const float* src, int a0) {
  if constexpr (N == 512 || N == 256) {
    fft_rows_half<N>(buf, twd, src, a0);
    __syncthreads();
  } else {
    fft_rows<N, F>(buf, twd, src, a0);
  }
}

// One transform pass: rows of `in` ([units][n][n]) -> orthonormal DST-I -> written transposed.
template <int N>
__global__ void __launch_bounds__(kThreads) k_dst_pass(const float* __restrict__ in, float* __restrict__ out,
                                                        const float2* __restrict__ tw) {
  constexpr int n = N - 1, L = 2 * N, F = kDstRows / 2;
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  float2* twd = smem2 + buf_elems<N>();
  const int u = blockIdx.y;
  const int a0 = blockIdx.x * kDstRows;
  const float* src = in + (size_t)u * n * n;
  for (int m = threadIdx.x; m < L; m += kThreads) twd[m] = tw[m];
  __syncthreads();
  fft_rows_any<N, F>(buf, twd, src, a0);
  // row pair (2f, 2f+1) packed as real + i imag: S x_{2f} = -Im Y / 2, S x_{2f+1} = Re Y / 2
  const float sc = 0.5f * sqrtf(2.0f / N);
  float* dst = out + (size_t)u * n * n;
  for (int idx = threadIdx.x; idx < n * kDstRows; idx += kThreads) {
    const int k = idx / kDstRows, r = idx - k * kDstRows;
    const int a = a0 + r;
    if (a >= n) continue;
    const float2 v = buf[(r >> 1) * buf_row<N>() + pad8(k + 1)];
    dst[(size_t)k * n + a] = (r & 1) ? v.x * sc : -v.y * sc;
  }
}

template <int N>
size_t dst_smem() {
  return (size_t)(buf_elems<N>() + 2 * N) * sizeof(float2);
}

// ------------------------------------------------------------------ FP64 stencils

__device__ __forceinline__ double lap5(const double* X, int n, int i, int j) {
  const double c = __ldcg(X + (size_t)i * n + j);
  const double w = (j > 0) ? __ldcg(X + (size_t)i * n + j - 1) : 0.0;
  const double e = (j < n - 1) ? __ldcg(X + (size_t)i * n + j + 1) : 0.0;
  const double s = (i > 0) ? __ldcg(X + (size_t)(i - 1) * n + j) : 0.0;
  const double no = (i < n - 1) ? __ldcg(X + (size_t)(i + 1) * n + j) : 0.0;
  return (w + e) + (s + no) - 4.0 * c;
}

// Right-hand side of Eq. 2.5: b = u + dt D_h v, v = u^3 - 3u (frozen model: v = -2u).
__device__ __forceinline__ double lin2_v(double u, int frozen) { return frozen ? -2.0 * u : u * u * u - 3.0 * u; }

// Block reduction (fixed tree): sum or min/max of doubles.
template <int OP>  // 0 sum, 1 max, 2 min
__device__ __forceinline__ double block_reduce(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (OP == 0) ? v + w : (OP == 1 ? fmax(v, w) : fmin(v, w));
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = sh[0];
  for (int i = 1; i < kThreads / 32; ++i) r = (OP == 0) ? r + sh[i] : (OP == 1 ? fmax(r, sh[i]) : fmin(r, sh[i]));
  return r;
}

// m(p,q) = 1/mu + e2dt mu + cdt wbar (diagonal of the preconditioner M in sine space). 1/mu by
// the correctly rounded reciprocal: the same value as the IEEE quotient 1.f / mu, without the
// division routine's slow-path call inside the epilogue loops.
__device__ __forceinline__ float mdiag(float mu, float e2dt, float cwb) { return __frcp_rn(mu) + e2dt * mu + cwb; }

// Start of a loop: counter = 0 and, for a nested loop, its condition = 1.
__global__ void k2_loop_start(cudaGraphConditionalHandle hnd, int* __restrict__ ctr, int which, int set_cond) {
  if (threadIdx.x == 0) {
    ctr[which] = 0;
    if (set_cond) cudaGraphSetConditional(hnd, 1u);
  }
}



template <typename K>
cudaError_t prep(K kernel, size_t smem) {
  static std::mutex mu;
  static std::set<std::pair<const void*, unsigned long long>> done;  // (kernel, context)
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(reinterpret_cast<const void*>(kernel), chctx::cache_key());
  if (done.count(key)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done.insert(key);
  return e;
}

template <int N>
cudaError_t dst_pass_n(const float* in, float* out, int units, const float2* tw, cudaStream_t st) {
  const size_t smem = dst_smem<N>();
  cudaError_t e = prep(k_dst_pass<N>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((N - 1 + kDstRows - 1) / kDstRows, units);
  k_dst_pass<N><<<grid, kThreads, smem, st>>>(in, out, tw);
  return cudaGetLastError();
}

cudaError_t dst_prepare(int n) {
  switch (n + 1) {
    case 16: return prep(k_dst_pass<16>, dst_smem<16>());
    case 32: return prep(k_dst_pass<32>, dst_smem<32>());
    case 64: return prep(k_dst_pass<64>, dst_smem<64>());
    case 128: return prep(k_dst_pass<128>, dst_smem<128>());
    case 256: return prep(k_dst_pass<256>, dst_smem<256>());
    case 512: return prep(k_dst_pass<512>, dst_smem<512>());
  }
  return cudaErrorInvalidValue;
}

cudaError_t dst_pass(int n, const float* in, float* out, int units, const float2* tw, cudaStream_t st) {
  switch (n + 1) {
    case 16: return dst_pass_n<16>(in, out, units, tw, st);
    case 32: return dst_pass_n<32>(in, out, units, tw, st);
    case 64: return dst_pass_n<64>(in, out, units, tw, st);
    case 128: return dst_pass_n<128>(in, out, units, tw, st);
    case 256: return dst_pass_n<256>(in, out, units, tw, st);
    case 512: return dst_pass_n<512>(in, out, units, tw, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

namespace {

// Parareal correction of one slice for every listed problem (Eq. 2.2), fused with the norms.
// Problem list entry i = problem index b; work row i of g / Wout.
//   init = 1: Unew = g (coarse initial guess); init = 0: Unew = F + (g - Gold), inc partial.
//   Gold = g; Wout (contiguous) = Unew; error partials against Uref (if given).
__global__ void k2_correct(double* __restrict__ U, const double* __restrict__ F, double* __restrict__ g,
                           double* __restrict__ Gold, const double* __restrict__ Uref, const int* __restrict__ list,
                           size_t pts, size_t ustride, size_t fstride, int init, double* __restrict__ part) {
  __shared__ double sh[kThreads / 32];
  const int i = blockIdx.y;
  const int b = list[i];
  double* Ub = U + (size_t)b * ustride;
  const double* Fb = F + (size_t)b * fstride;
  double* Gb = Gold + (size_t)b * fstride;
  double* gi = g + (size_t)i * pts;
  double inc = 0.0, e2 = 0.0, em = 0.0, um = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < pts; k += (size_t)gridDim.x * blockDim.x) {
    const double gv = gi[k];
    const double nw = init ? gv : Fb[k] + (gv - Gb[k]);
    if (!init) inc = fmax(inc, fabs(nw - Ub[k]));
    um = isfinite(nw) ? fmax(um, fabs(nw)) : INFINITY;
    Ub[k] = nw;
    Gb[k] = gv;
    gi[k] = nw;
    if (Uref) {
      const double e = nw - Uref[(size_t)b * ustride + k];
      e2 += e * e;
      em = fmax(em, fabs(e));
    }
  }
  const double r0 = block_reduce<1>(inc, sh);
  const double r1 = block_reduce<0>(e2, sh);
  const double r2 = block_reduce<1>(em, sh);
  const double r3 = block_reduce<1>(um, sh);
  if (threadIdx.x == 0) {
    part[((size_t)i * 4 + 0) * kBlk + blockIdx.x] = r0;
    part[((size_t)i * 4 + 1) * kBlk + blockIdx.x] = r1;
    part[((size_t)i * 4 + 2) * kBlk + blockIdx.x] = r2;
    part[((size_t)i * 4 + 3) * kBlk + blockIdx.x] = r3;
  }
}

// Fold the slice's partials into per-problem running maxima acc[b] = {inc, err_l2, err_max}.
__global__ void k2_correct_fold(const double* __restrict__ part, const int* __restrict__ list, int count,
                                double* __restrict__ acc, double h2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double inc = 0.0, e2 = 0.0, em = 0.0, um = 0.0;
  for (int k = 0; k < kBlk; ++k) {
    inc = fmax(inc, part[((size_t)i * 4 + 0) * kBlk + k]);
    e2 += part[((size_t)i * 4 + 1) * kBlk + k];
    em = fmax(em, part[((size_t)i * 4 + 2) * kBlk + k]);
    um = fmax(um, part[((size_t)i * 4 + 3) * kBlk + k]);
  }
  const int b = list[i];
  acc[b * 4 + 0] = fmax(acc[b * 4 + 0], inc);
  acc[b * 4 + 1] = fmax(acc[b * 4 + 1], sqrt(h2 * e2));
  acc[b * 4 + 2] = fmax(acc[b * 4 + 2], em);
  acc[b * 4 + 3] = fmax(acc[b * 4 + 3], um);
}

// Gather rows: dst[i] = src + off[i] (element offsets), pts each.
__global__ void k2_gather(double* __restrict__ dst, const double* __restrict__ src, const long long* __restrict__ off,
                          size_t pts) {
  const int i = blockIdx.y;
  const double* s = src + off[i];
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < pts; k += (size_t)gridDim.x * blockDim.x)
    dst[(size_t)i * pts + k] = s[k];
}
__global__ void k2_scatter(double* __restrict__ dst, const double* __restrict__ src, const long long* __restrict__ off,
                           size_t pts) {
  const int i = blockIdx.y;
  double* d = dst + off[i];
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < pts; k += (size_t)gridDim.x * blockDim.x)
    d[k] = src[(size_t)i * pts + k];
}

}  // namespace

cudaError_t launch_correct(double* U, const double* F, double* g, double* Gold, const double* Uref, const int* list,
                           int count, size_t pts, size_t ustride, size_t fstride, int init, double* part, double* acc,
                           double h2, cudaStream_t st) {
  if (count < 1) return cudaSuccess;
  k2_correct<<<dim3(kBlk, count), kThreads, 0, st>>>(U, F, g, Gold, Uref, list, pts, ustride, fstride, init, part);
  k2_correct_fold<<<(count + 127) / 128, 128, 0, st>>>(part, list, count, acc, h2);
  return cudaGetLastError();
}

cudaError_t launch_gather(double* dst, const double* src, const long long* off, int count, size_t pts, cudaStream_t st) {
  if (count < 1) return cudaSuccess;
  k2_gather<<<dim3(kBlk, count), kThreads, 0, st>>>(dst, src, off, pts);
  return cudaGetLastError();
}

cudaError_t launch_scatter(double* dst, const double* src, const long long* off, int count, size_t pts,
                           cudaStream_t st) {
  if (count < 1) return cudaSuccess;
  k2_scatter<<<dim3(kBlk, count), kThreads, 0, st>>>(dst, src, off, pts);
  return cudaGetLastError();
}

size_t correct_partials(int count) { return (size_t)count * 4 * kBlk; }

// ---------------------------------------------------------------------------- Prop2D

// Twiddles of the stages after the first of fft_rows<N> (radix 8 with Ns = 8, 64, ..., then the
// radix-2 or radix-4 stage), stage after stage: entry (r - 1) Ns + k = exp(-2 pi i m / L) with
// m = r k L / (R Ns), r = 1..R-1, k < Ns (host libm, rounded to FP32). At most L entries. For
// N = 512 and 256 the tables of fft512_warp / fft256_warp and the sines of fft_rows_half.
static std::vector<float2> twiddle_table(int N) {
  const int L = 2 * N;
  if (N == 512 || N == 256) {  // N-point warp FFT: tw2[k1][t] = exp(-2 pi i k1 t / N), t < 32
    std::vector<float2> tw(L, make_float2(0.f, 0.f));
    for (int k1 = 0; k1 < N / 32; ++k1)
      for (int t = 0; t < 32; ++t) {
        const double a = -2.0 * M_PI * k1 * t / N;
        tw[k1 * 32 + t] = make_float2(float(std::cos(a)), float(std::sin(a)));
      }
    float* sj = reinterpret_cast<float*>(tw.data() + N);  // then sin(pi j / N), j < N (fft_rows_half)
    for (int j = 0; j < N; ++j) sj[j] = float(std::sin(M_PI * j / N));
    return tw;
  }
  int lg = 0;
  while ((1 << lg) < L) ++lg;
  const int n8 = lg / 3, rem = lg - 3 * n8;
  std::vector<float2> tw;
  auto stage = [&](int R, int Ns) {
    for (int r = 1; r < R; ++r)
      for (int k = 0; k < Ns; ++k) {
        const long long m = (long long)r * k * (L / (R * Ns));
        tw.push_back(make_float2(float(std::cos(-2.0 * M_PI * m / L)), float(std::sin(-2.0 * M_PI * m / L))));
      }
  };
  int Ns = 8;
  for (int s = 1; s < n8; ++s, Ns *= 8) stage(8, Ns);
  if (rem == 1) stage(2, Ns);
  if (rem == 2) stage(4, Ns);
  tw.resize(L, make_float2(0.f, 0.f));
  return tw;
}

cudaError_t Prop2D::init(const Params2D& p, int cap, cudaStream_t st) {
  if (!supported_n(p.n) || cap < 1) return cudaErrorInvalidValue;
  // CH_2D_STEP=persistent | host selects another execution of the same phases (default: graphs)
  const char* env = std::getenv("CH_2D_STEP");
  path_ = PATH_GRAPH;
  if (env && std::strcmp(env, "persistent") == 0) path_ = PATH_PERSISTENT;
  if (env && std::strcmp(env, "host") == 0) path_ = PATH_HOST;
  if (env && std::strcmp(env, "cluster") == 0) path_ = PATH_CLUSTER;
  const char* cl = std::getenv("CH_2D_CLUSTER");  // cluster size of the cluster execution (default: chosen)
  cluster_force_ = cl ? std::atoi(cl) : 0;
  const char* mb = std::getenv("CH_2D_MINB");
  persist_minb_ = mb ? std::atoi(mb) : 3;
  p_ = p;
  cap_ = cap;
  pts_ = (size_t)p.n * p.n;
  nblk_ = kBlk;
  const size_t v64 = (size_t)cap * pts_ * sizeof(double), v32 = (size_t)cap * pts_ * sizeof(float);
  cudaError_t e = cudaSuccess;
  auto al = [&](void** ptr, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, b);
    bytes_ += b;
  };
  al((void**)&yhat_, v64);
  al((void**)&yprev_, v64);
  al((void**)&z_, v64);
  al((void**)&xacc_, v64);
  al((void**)&w_, v32);
  al((void**)&rhs_, v32);
  al((void**)&xh_, v32);
  al((void**)&rh_, v32);
  al((void**)&ph_, v32);
  al((void**)&qh_, v32);
  al((void**)&tmp_, v32);
  al((void**)&tmp2_, v32);
  al((void**)&mu_, p.n * sizeof(float));
  al((void**)&tw_, (size_t)2 * (p.n + 1) * sizeof(float2));
  al((void**)&part_, (size_t)cap * 2 * kBlk * sizeof(double));
  al((void**)&scal_, (size_t)cap * 8 * sizeof(double));
  al((void**)&flag_, (size_t)cap * 2 * sizeof(int));
  al((void**)&newton_cnt_, (size_t)cap * sizeof(int));
  al((void**)&status_, 4 * sizeof(unsigned) + sizeof(unsigned long long));
  al((void**)&ctr_, 4 * kMaxGroups * sizeof(int));
  // [0] CG iterations (batched), [1] Newton passes (batched), [2] CG iterations summed over units
  al((void**)&cg_dev_, 4 * sizeof(unsigned long long));
  al((void**)&ppart_, (size_t)7 * cap * ((p.n + kDstRows - 1) / kDstRows) * sizeof(double));
  al((void**)&active_, 4 * kMaxGroups * sizeof(int));
  al((void**)&cgs_, (size_t)cap * 8 * sizeof(double));
  al((void**)&uh_, v32);
  al((void**)&sh_, v32);
  al((void**)&bar_, 4 * sizeof(unsigned));
  if (e != cudaSuccess) return e;
  e = cudaHostAlloc((void**)&host_cnt_, 8 * sizeof(int), 0);
  if (e != cudaSuccess) return e;
  if ((e = dst_prepare(p.n)) != cudaSuccess) return e;  // kernel attributes, before any capture
  // eigenvalues of A = -D_1: mu_p = (4/h^2) sin^2(p pi / (2(n+1))), p = 1..n (host libm)
  std::vector<float> mu(p.n);
  for (int q = 1; q <= p.n; ++q) {
    const double s = std::sin(q * M_PI / (2.0 * (p.n + 1)));
    mu[q - 1] = float(4.0 / (p.h * p.h) * s * s);
  }
  const std::vector<float2> tw = twiddle_table(p.n + 1);
  e = cudaMemcpyAsync(mu_, mu.data(), mu.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tw_, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status_, 0, 4 * sizeof(unsigned) + sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cg_dev_, 0, 4 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctr_, 0, 4 * kMaxGroups * sizeof(int), st);  // [2], [3]: scalar kernels
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

void Prop2D::release() {
  for (auto& c : graphs_) cudaGraphExecDestroy(c.second);
  graphs_.clear();
  for (int g = 0; g < kMaxGroups; ++g) {
    if (gs_[g]) cudaStreamDestroy(gs_[g]);
    if (gev_[g]) cudaEventDestroy(gev_[g]);
    gs_[g] = nullptr;
    gev_[g] = nullptr;
  }
  if (gfork_) cudaEventDestroy(gfork_);
  gfork_ = nullptr;
  void* ptrs[] = {yhat_, yprev_, z_, xacc_, w_, rhs_, xh_, rh_, ph_, qh_, tmp_, tmp2_, mu_, tw_, part_, scal_, flag_,
                  newton_cnt_, status_, ctr_, cg_dev_, ppart_, active_, bar_, cgs_, uh_, sh_};
  for (void* q : ptrs) cudaFree(q);
  if (host_cnt_) cudaFreeHost(host_cnt_);
  host_cnt_ = nullptr;
  yhat_ = yprev_ = z_ = xacc_ = nullptr;
  w_ = rhs_ = xh_ = rh_ = ph_ = qh_ = tmp_ = tmp2_ = mu_ = nullptr;
  tw_ = nullptr;
  part_ = scal_ = nullptr;
  flag_ = newton_cnt_ = ctr_ = nullptr;
  status_ = nullptr;
  cg_dev_ = nullptr;
  ppart_ = nullptr;
  active_ = nullptr;
  bar_ = nullptr;
  cgs_ = nullptr;
  uh_ = sh_ = nullptr;
}

cudaError_t Prop2D::dst2(const float* in, float* out, int units, cudaStream_t st) {
  cudaError_t e = dst_pass(p_.n, in, tmp2_ == out ? tmp_ : tmp2_, units, tw_, st);
  if (e == cudaSuccess) e = dst_pass(p_.n, tmp2_ == out ? tmp_ : tmp2_, out, units, tw_, st);
  return e;
}


namespace {

// Adds a WHILE node at the current capture position of `st` and returns its body graph.
cudaError_t add_while(cudaStream_t st, cudaGraphConditionalHandle* hnd, unsigned dflt, unsigned flags,
                      cudaGraph_t* body) {
  cudaStreamCaptureStatus stt;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &stt, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (hnd && !*hnd) {
    e = cudaGraphConditionalHandleCreate(hnd, g, dflt, flags);
    if (e != cudaSuccess) return e;
  }
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = *hnd;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Current capture graph of a stream (to create a handle before the node that uses it).
cudaError_t capture_graph(cudaStream_t st, cudaGraph_t* g) {
  cudaStreamCaptureStatus stt;
  return cudaStreamGetCaptureInfo(st, &stt, nullptr, g, nullptr, nullptr, nullptr);
}

}  // namespace

// Captures one implicit step of the batch as a graph: the right-hand side kernels, then a
// device-driven Newton loop whose body forms the FP64 residual, runs a device-driven CG loop
// in sine space and applies the correction. Nothing returns to the host inside the step.
cudaError_t Prop2D::propagate(double* Y, int units, int scheme, double dt, int nsteps, cudaStream_t st) {
  if (units > cap_ || units < 1) return cudaErrorInvalidValue;
  if (path_ == PATH_PERSISTENT) return propagate_persistent(Y, units, scheme, dt, nsteps, st);
  if (path_ == PATH_CLUSTER) return propagate_cluster(Y, units, scheme, dt, nsteps, st);
  if (path_ == PATH_HOST) return propagate_host(Y, units, scheme, dt, nsteps, st);
  // Independent units are split into up to kMaxGroups groups whose step graphs run concurrently
  // on streams of their own: each phase is a chain of dependent latencies over few blocks, so
  // concurrent groups fill the GPU that one group leaves idle.
  int groups = std::max(1, std::min(kMaxGroups, units / kMinGroupUnits));
  if (const char* ge = std::getenv("CH_2D_GROUPS")) groups = std::max(1, std::min(groups, std::atoi(ge)));
  cudaError_t e = cudaSuccess;
  if (groups > 1) {
    if (!gs_[0]) {
      for (int g = 0; g < kMaxGroups && e == cudaSuccess; ++g) {
        e = cudaStreamCreateWithFlags(&gs_[g], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&gev_[g], cudaEventDisableTiming);
      }
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&gfork_, cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
    if ((e = cudaEventRecord(gfork_, st)) != cudaSuccess) return e;
  }
  for (int g = 0; g < groups && groups > 1; ++g)
    if ((e = cudaStreamWaitEvent(gs_[g], gfork_, 0)) != cudaSuccess) return e;
  // step j of every group, then step j + 1: the groups' graphs are enqueued side by side
  for (int j = 0; j < nsteps; ++j) {
    for (int g = 0; g < groups; ++g) {
      const int u0 = (int)((long long)units * g / groups), u1 = (int)((long long)units * (g + 1) / groups);
      cudaStream_t gst = (groups > 1) ? gs_[g] : st;
      StepKey k{Y + (size_t)u0 * pts_, u1 - u0, scheme, dt, (scheme == SCHEME_NL && j > 0) ? 1 : 0, u0, g};
      cudaGraphExec_t ex = nullptr;
      for (auto& c : graphs_)
        if (c.first == k) ex = c.second;
      if (!ex) {
        if ((e = build_step(k, &ex)) != cudaSuccess) return e;
        graphs_.push_back({k, ex});
      }
      if ((e = cudaGraphLaunch(ex, gst)) != cudaSuccess) return e;
      step_kernels_ += (scheme == SCHEME_NL) ? kStepKernelsNL : kStepKernelsLin;
    }
  }
  for (int g = 0; g < groups && groups > 1; ++g) {
    if ((e = cudaEventRecord(gev_[g], gs_[g])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, gev_[g], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t Prop2D::reset_counters(cudaStream_t st) {
  newton_total_ = 0;
  newton_peak_ = 0;
  cg_total_ = 0;
  cudaError_t e = cudaMemsetAsync(status_, 0, 4 * sizeof(unsigned) + sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cg_dev_, 0, 4 * sizeof(unsigned long long), st);
  return e;
}

__global__ void k2_clear_status(unsigned* status, unsigned mask) { atomicAnd(status, ~mask); }

cudaError_t Prop2D::clear_status(unsigned mask, cudaStream_t st) {
  k2_clear_status<<<1, 1, 0, st>>>(status_, mask);
  return cudaGetLastError();
}

unsigned Prop2D::read_status(cudaStream_t st) {
  unsigned s[4] = {0, 0, 0, 0};
  unsigned long long tot = 0;
  cudaMemcpyAsync(s, status_, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&tot, (int*)status_ + 4, sizeof(tot), cudaMemcpyDeviceToHost, st);
  unsigned long long cgt[4] = {0, 0, 0, 0};
  cudaMemcpyAsync(cgt, cg_dev_, sizeof(cgt), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  cg_total_ = (long long)cgt[0];
  newton_passes_ = (long long)cgt[1];
  cg_unit_total_ = (long long)cgt[2];
  newton_total_ = tot;
  newton_peak_ = (int)s[3];
  return s[0];
}

// ------------------------------------------------------------------ persistent fine sweep
//
// The whole propagation (nsteps implicit steps, each an FP64 Newton loop around FP32 CG in sine
// space) as one cooperative kernel. Work items are (unit, block of kDstRows rows); every phase
// below is a loop of the grid's blocks over the items of the units that are still active,
// and phases are separated by a grid barrier (all blocks are co-resident: cooperative launch).
// The transform passes carry the pointwise work of the graph path in their epilogues. Loop
// exits are decided from counters read after a barrier, so every block takes the same
// branches; a barrier that waits too long sets ST_TIMEOUT and every block returns.
// Arguments of the step phases (shared by the graph and the persistent execution).
struct PArgs {
  double* Y;
  double* yhat;
  double* yprev;
  double* z;
  float* w;
  float* rhs;
  float* xh;
  float* rh;
  float* ph;
  float* qh;
  float* tmp;
  float* t2;
  const float* mu1;
  const float2* tw;
  double* pmin;   // [units][nb] per item: min wc
  double* pmax;   //                 max wc
  double* pdel;   //                 (w, u)
  double* cgs;    // [units][8]      CG scalars: alpha, gamma of the last iteration (parity
                  //                 slots 0, 1 and 2, 3), gamma_0 (slot 4), beta (parity
                  //                 slots 5, 6)
  float* uh;      // u = M^{-1} r (sine space)
  float* sh;      // s = S p (sine space)
  double* pgam;   // [units][nb]     (r, u)
  double* pd;     // [units][nb]     max |d|
  int* flag;      // [units][2]: Newton done, CG done
  int* cnt;       // [units] Newton iterations of the step
  double* scal;   // [units][8]: [4] wbar of the Newton iteration, [6] previous max |d|
  unsigned* status;
  unsigned long long* totals;  // [0] batched CG iterations, [1] batched Newton passes
  int* active;    // [0..1] CG, [2..3] Newton: units still iterating (parity slots)
  unsigned* bar;  // [0] arrivals, [1] generation, [2] abort
  int* ctr;       // graph path: [0] Newton, [1] CG iteration of the loop being replayed
  const double* W64;
  double wconst, dt, ih2, c1, tol, floor_, cg_tol2;
  float fe2dt, fdt;
  double eps2;           // eps^2 of every unit, unless eps2u is set
  const double* eps2u;   // per-unit eps^2 [units] (device) or null
  int units, nsteps, scheme, zmode, newton_max, cg_max, have_prev0, frozen;
  cudaGraphConditionalHandle hcg;  // graph path, small batches: the CG loop's condition (PH_P4S)
};

namespace {

constexpr unsigned kBarrierSpins = 1u << 22;  // x ~0.5 us sleeps: a stuck barrier gives up in ~2 s


__device__ __forceinline__ bool grid_barrier(unsigned* bar) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = bar + 1;
    volatile unsigned* abort_ = bar + 2;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned spins = 0;
      while (*gen == g) {
        if (*abort_ || ++spins > kBarrierSpins) {
          ok = 0;
          atomicExch(bar + 2, 1u);
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Work items (unit, block of kDstRows rows) that a block walks in a phase: first, first + step,
// ... below end. chk = 1: units whose Newton loop (and, for the CG phases, CG loop) has ended are
// skipped, read from the per-unit flags (batched executions); chk = 0: no test (the cluster
// execution, whose loops end per unit).
struct Items {
  int first, step, end, chk;
};

template <int N>
__device__ __forceinline__ Items grid_items(const PArgs& a) {
  constexpr int nb = (N - 1 + kDstRows - 1) / kDstRows;
  return Items{(int)blockIdx.x, (int)gridDim.x, a.units * nb, 1};
}

// Per-unit scalars from the nb per-item partials. Partials are read with L2-coherent loads (in
// the persistent and cluster executions other blocks of the same kernel wrote them). The block
// versions are formed by the first warp (lane b holds partial b, a fixed shuffle tree) and handed
// to every thread through shared memory: the same reduction in all threads would queue the whole
// block on GB300's narrow FP64 pipe. They synchronise the block: call them from block-uniform
// code only.
template <int N>
__device__ __forceinline__ double unit_wbar(const PArgs& a, int u) {
  constexpr int nb = (N - 1 + kDstRows - 1) / kDstRows;
  static_assert(nb <= 32, "one partial per lane");
  __shared__ double res;
  __syncthreads();  // earlier readers of res are done
  if (threadIdx.x < 32) {
    double lo = 1e300, hi = -1e300;
    if (threadIdx.x < nb) {
      lo = __ldcg(a.pmin + (size_t)u * nb + threadIdx.x);
      hi = __ldcg(a.pmax + (size_t)u * nb + threadIdx.x);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (threadIdx.x == 0) res = 0.5 * (lo + hi);
  }
  __syncthreads();
  return res;
}

// OP 0: sum of the partials; 1: their maximum (and 0).
template <int N, int OP>
__device__ __forceinline__ double unit_reduce(const double* p, int u) {
  constexpr int nb = (N - 1 + kDstRows - 1) / kDstRows;
  static_assert(nb <= 32, "one partial per lane");
  __shared__ double res;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < nb) ? __ldcg(p + (size_t)u * nb + threadIdx.x) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v, o);
      v = (OP == 0) ? v + w : fmax(v, w);
    }
    if (threadIdx.x == 0) res = v;
  }
  __syncthreads();
  return res;
}

// Maximum of the partials (and 0) in the calling thread alone.
template <int N>
__device__ __forceinline__ double unit_max_thread(const double* p, int u) {
  constexpr int nb = (N - 1 + kDstRows - 1) / kDstRows;
  double m = 0.0;
  for (int b = 0; b < nb; ++b) m = fmax(m, __ldcg(p + (size_t)u * nb + b));
  return m;
}


// Calls f as a separate function: the persistent kernel's register allocation is then that of
// its largest phase, not of all phases inlined together.
template <typename F>
__device__ __noinline__ void noinl(const F& f) {
  f();
}

// eps^2 dt of unit u (FP32 for the sine-space solver) and c1 = eps^2 dt / h^2 (FP64 residual).
__device__ __forceinline__ float unit_fe2dt(const PArgs& a, int u) {
  return a.eps2u ? float(a.eps2u[u] * a.dt) : a.fe2dt;
}
__device__ __forceinline__ double unit_c1(const PArgs& a, int u) { return a.eps2u ? a.eps2u[u] * a.dt * a.ih2 : a.c1; }

enum Epi { E_PLAIN = 0, E_WPROD, E_W, E_INIT, E_UPDATE };

// One transform pass over the items of active units: rows [a0, a0 + kDstRows) of `in` ->
// DST-I -> column a of the output (transposed), then the epilogue.
//   E_PLAIN: out = v;  E_WPROD: out = dt (wc - wbar) v;  E_W: w = m u + v (= S u), sums (w, u)
//   and (r, u);  E_INIT: r = v / mu, u = r / m, x = 0;  E_UPDATE: Y -= v, max |v|.
// `act` selects the units: 0 = not Newton-done, 1 = not Newton-done and not CG-done; -1 = no
// test, and wb is the unit's wbar (otherwise it is formed from the range partials).
// Epilogue loads of arrays written earlier in the kernel are L2-coherent.
template <int N, int EPI>
__device__ __forceinline__ void dst_item(const PArgs& a, float2* buf, const float2* twd, const float* in, float* out,
                                         int act, double* part, int item, double wb = 0.0) {
  constexpr int n = N - 1, nb = (n + kDstRows - 1) / kDstRows;
  static_assert(kThreads % kDstRows == 0, "epilogue thread layout");
  constexpr int KS = kThreads / kDstRows;  // output rows apart of one thread's elements
  constexpr int J = (n + KS - 1) / KS;     // epilogue elements per thread
  constexpr int UBM = (EPI == E_W || EPI == E_UPDATE) ? 8 : 16;  // two operands, or an FP64 one
  constexpr int UB = J < UBM ? J : UBM;       // elements whose loads are issued together
  static_assert(J % UB == 0, "epilogue batches");
  __shared__ double sh[kThreads / 32];
  const size_t pts = (size_t)n * n;
  const float sc = 0.5f * sqrtf(2.0f / N);
  const float* __restrict__ mu1 = a.mu1;
  const int u = item / nb, b = item - u * nb, a0 = b * kDstRows;
  if (act >= 0 && (a.flag[2 * u] || (act == 1 && a.flag[2 * u + 1]))) return;  // block-uniform
  fft_rows_any<N, kDstRows / 2>(buf, twd, in + u * pts, a0);
  float cwb = 0.f;
  // wbar: formed from the range partials in the CG-start pass, which keeps it for the CG passes
  if (act >= 0 && EPI == E_INIT) {
    wb = unit_wbar<N>(a, u);
    if (b == 0 && threadIdx.x == 0) a.scal[u * 8 + 4] = wb;
  } else if (act >= 0 && (EPI == E_WPROD || EPI == E_W)) {
    wb = __ldcg(a.scal + u * 8 + 4);
  }
  if (EPI == E_WPROD || EPI == E_W || EPI == E_INIT) cwb = float(wb);
  const float fcwb = a.fdt * cwb;
  const float fe2dt = unit_fe2dt(a, u);
  // This thread's outputs: column c = a0 + r of the rows k = k0, k0 + KS, ... (row pair
  // (2f, 2f+1) was packed as real + i imag: S x_{2f} = -Im Y / 2, S x_{2f+1} = Re Y / 2).
  const int r = threadIdx.x % kDstRows, k0 = threadIdx.x / kDstRows, c = a0 + r;
  const bool cok = c < n;
  const float mc = mu1[cok ? c : 0];
  const size_t ob = u * pts + c;
  // per-thread partial sums / maxima in FP32 (GB300's FP64 pipe is 1/64 of FP32), combined across
  // the block in FP64
  float acc = 0.f, acc2 = 0.f;
  bool bad = false;
#pragma unroll 1
  for (int j0 = 0; j0 < J; j0 += UB) {
    float v[UB], ld[UB], ld2[UB];
    double yv[UB];
#pragma unroll
    for (int q = 0; q < UB; ++q) {
      const int k = k0 + (j0 + q) * KS;
      v[q] = ld[q] = ld2[q] = 0.f;
      yv[q] = 0.0;
      if (cok && k < n) {
        const size_t o = ob + (size_t)k * n;
        if (EPI == E_WPROD) ld[q] = __ldcg(a.w + o);
        if (EPI == E_W) {
          ld[q] = __ldcg(a.uh + o);
          ld2[q] = __ldcg(a.rh + o);
        }
        if (EPI == E_UPDATE) yv[q] = __ldcg(a.Y + o);
        const float2 cv = buf[(r >> 1) * buf_row<N>() + pad8(k + 1)];
        v[q] = (r & 1) ? cv.x * sc : -cv.y * sc;
      }
    }
#pragma unroll
    for (int q = 0; q < UB; ++q) {
      const int k = k0 + (j0 + q) * KS;
      if (!(cok && k < n)) continue;
      const size_t o = ob + (size_t)k * n;
      if (EPI == E_PLAIN) {
        out[o] = v[q];
      } else if (EPI == E_WPROD) {
        out[o] = a.fdt * (ld[q] - cwb) * v[q];
      } else if (EPI == E_W) {
        const float w = mdiag(mu1[k] + mc, fe2dt, fcwb) * ld[q] + v[q];
        a.qh[o] = w;
        acc = fmaf(w, ld[q], acc);
        acc2 = fmaf(ld2[q], ld[q], acc2);
      } else if (EPI == E_INIT) {
        const float mu = mu1[k] + mc;
        const float r0 = v[q] / mu;
        a.xh[o] = 0.f;
        a.rh[o] = r0;
        a.uh[o] = r0 * __frcp_rn(mdiag(mu, fe2dt, fcwb));
      } else {  // E_UPDATE
        bad |= !isfinite(v[q]);
        a.Y[o] = yv[q] - (double)v[q];
        acc = fmaxf(acc, fabsf(v[q]));
      }
    }
  }
  if (EPI == E_UPDATE) {
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, ST_NONFINITE);
    const double m = block_reduce<1>((double)acc, sh);
    if (threadIdx.x == 0) part[(size_t)u * nb + b] = m;
  } else if (EPI == E_W) {
    // FP32 shuffle tree within each warp, the warps' sums added in FP64 in a fixed order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_xor_sync(0xffffffffu, acc, o);
      acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
    }
    __shared__ float ws[2][kThreads / 32];
    if ((threadIdx.x & 31) == 0) {
      ws[0][threadIdx.x >> 5] = acc;
      ws[1][threadIdx.x >> 5] = acc2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double wu = 0.0, ru = 0.0;
      for (int i = 0; i < kThreads / 32; ++i) {
        wu += (double)ws[0][i];
        ru += (double)ws[1][i];
      }
      a.pdel[(size_t)u * nb + b] = wu;
      a.pgam[(size_t)u * nb + b] = ru;
    }
  }
}

// A transform phase of the persistent kernel: its blocks walk the items (one call per item keeps
// the transform's register allocation that of a single item).
template <int N, int EPI>
__device__ __forceinline__ void dst_phase(const PArgs& a, float2* buf, const float2* twd, const float* in, float* out,
                                          int act, double* part) {
  constexpr int nb = (N - 1 + kDstRows - 1) / kDstRows;
  for (int item = blockIdx.x; item < a.units * nb; item += gridDim.x) {
    __syncthreads();  // the previous item's epilogue has finished reading buf
    noinl([&] { dst_item<N, EPI>(a, buf, twd, in, out, act, part, item); });
  }
}

// Rows [a0, a0 + kDstRows) of unit u, element e of the item: (i, j), or false past the grid.
template <int N>
__device__ __forceinline__ bool item_elem(int a0, int e, int& i, int& j) {
  constexpr int n = N - 1;
  i = a0 + e / n;
  j = e - (e / n) * n;
  return i < n;
}

// The phases of the persistent kernel, each compiled as its own function (keeps the kernel's
// register allocation to that of its largest phase). `a` lives in shared memory.
template <int N>
__device__ __forceinline__ void ph_prologue_items(const PArgs& a, Items its) {
  constexpr int n = N - 1, nb = (n + kDstRows - 1) / kDstRows;
  const size_t pts = (size_t)n * n;
  for (int item = its.first; item < its.end; item += its.step) {
    const int u = item / nb, a0 = (item - u * nb) * kDstRows;
    const double* Yu = a.Y + u * pts;
#pragma unroll 1
    for (int e = threadIdx.x; e < kDstRows * n; e += kThreads) {
      int i, j;
      if (!item_elem<N>(a0, e, i, j)) continue;
      const size_t k = (size_t)i * n + j;
      const double yk = __ldcg(Yu + k);
      if (a.scheme == SCHEME_NL) {
        a.yhat[u * pts + k] = yk - a.dt * a.ih2 * lap5(Yu, n, i, j);
      } else {
        a.yprev[u * pts + k] = yk;
        if (a.scheme == SCHEME_LIN1) {
          a.yhat[u * pts + k] = yk - a.dt * a.ih2 * lap5(Yu, n, i, j);
        } else {
          const double c = lin2_v(yk, a.frozen);
          const double w_ = (j > 0) ? lin2_v(__ldcg(Yu + k - 1), a.frozen) : 0.0;
          const double e_ = (j < n - 1) ? lin2_v(__ldcg(Yu + k + 1), a.frozen) : 0.0;
          const double s_ = (i > 0) ? lin2_v(__ldcg(Yu + k - n), a.frozen) : 0.0;
          const double no = (i < n - 1) ? lin2_v(__ldcg(Yu + k + n), a.frozen) : 0.0;
          a.yhat[u * pts + k] = yk + a.dt * a.ih2 * ((w_ + e_) + (s_ + no) - 4.0 * c);
        }
      }
    }
  }
}

template <int N>
__device__ __forceinline__ void ph_prologue(const PArgs& a, int step) {
  (void)step;
  ph_prologue_items<N>(a, grid_items<N>(a));
  for (int u = blockIdx.x * kThreads + threadIdx.x; u < a.units; u += gridDim.x * kThreads) {
    a.flag[2 * u] = 0;
    a.flag[2 * u + 1] = 0;
    a.cnt[u] = 0;
    a.scal[u * 8 + 6] = 0.0;
  }
}

template <int N>
__device__ __forceinline__ void ph_predict(const PArgs& a, int have_prev) {
  constexpr int n = N - 1;
  const size_t total = (size_t)a.units * n * n;
  if (a.scheme == SCHEME_NL)
    for (size_t k = blockIdx.x * (size_t)kThreads + threadIdx.x; k < total; k += (size_t)gridDim.x * kThreads) {
      const double y = a.Y[k];
      const double g = have_prev ? 2.0 * y - a.yprev[k] : y;
      a.yprev[k] = y;
      a.Y[k] = g;
    }
  if (blockIdx.x == 0 && threadIdx.x < 4) a.active[threadIdx.x] = 0;
}

// The predictor over the rows of the given items (the cluster execution).
template <int N>
__device__ __forceinline__ void ph_predict_items(const PArgs& a, int have_prev, Items its) {
  constexpr int n = N - 1, nb = (n + kDstRows - 1) / kDstRows;
  const size_t pts = (size_t)n * n;
  if (a.scheme != SCHEME_NL) return;
  for (int item = its.first; item < its.end; item += its.step) {
    const int u = item / nb, a0 = (item - u * nb) * kDstRows;
    const size_t base = u * pts + (size_t)a0 * n;
    const int cnt = (n - a0 < kDstRows ? n - a0 : kDstRows) * n;
    for (int e = threadIdx.x; e < cnt; e += kThreads) {
      const double y = __ldcg(a.Y + base + e);
      const double g = have_prev ? 2.0 * y - __ldcg(a.yprev + base + e) : y;
      a.yprev[base + e] = y;
      a.Y[base + e] = g;
    }
  }
}

// Five-point Laplacian of X at (i, j) of an n x n grid (zero outside), restrict loads.
template <int n>
__device__ __forceinline__ double lap5r(const double* __restrict__ X, int i, int j) {
  const size_t k = (size_t)i * n + j;
  const double c = __ldcg(X + k);
  const double w = (j > 0) ? __ldcg(X + k - 1) : 0.0;
  const double e = (j < n - 1) ? __ldcg(X + k + 1) : 0.0;
  const double s = (i > 0) ? __ldcg(X + k - n) : 0.0;
  const double no = (i < n - 1) ? __ldcg(X + k + n) : 0.0;
  return (w + e) + (s + no) - 4.0 * c;
}

// Sum of the four neighbours of X at (i, j) (zero outside), restrict loads; c = X(i, j).
template <int n>
__device__ __forceinline__ double nsum4r(const double* __restrict__ X, int i, int j, double& c) {
  const size_t k = (size_t)i * n + j;
  c = __ldcg(X + k);
  const double w = (j > 0) ? __ldcg(X + k - 1) : 0.0;
  const double e = (j < n - 1) ? __ldcg(X + k + 1) : 0.0;
  const double s = (i > 0) ? __ldcg(X + k - n) : 0.0;
  const double no = (i < n - 1) ? __ldcg(X + k + n) : 0.0;
  return (w + e) + (s + no);
}

// N1: z = (c1 lap(Y) - dt g(Y)) / h^2, formed as c1' S4(Y) + Y (-4 c1' - dt' g(Y) / Y) with the
// neighbour sum S4, c1' = c1 / h^2, dt' = dt / h^2: seven FP64 operations per node on GB300's
// narrow FP64 pipe (the 1/h^2 of the residual's Laplacian is folded in here).
template <int N>
__device__ __forceinline__ void ph_z(const PArgs& a, Items its) {
  constexpr int n = N - 1, nb = (n + kDstRows - 1) / kDstRows, U = 4;
  const size_t pts = (size_t)n * n;
  double* __restrict__ z = a.z;
  const double* __restrict__ W64 = a.W64;
  for (int item = its.first; item < its.end; item += its.step) {
    const int u = item / nb, a0 = (item - u * nb) * kDstRows;
    if (its.chk && a.flag[2 * u]) continue;
    const double* __restrict__ Yu = a.Y + u * pts;
    const int cnt = (n - a0 < kDstRows ? n - a0 : kDstRows) * n;
    const double c1s = unit_c1(a, u) * a.ih2, m4c1s = -4.0 * c1s, dts = a.dt * a.ih2;
    for (int e0 = threadIdx.x; e0 < cnt; e0 += U * kThreads) {
      double sv[U], xv[U], wv[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int e = e0 + q * kThreads;
        if (e < cnt) {
          const int i = a0 + e / n, j = e - (e / n) * n;
          const size_t k = (size_t)i * n + j;
          sv[q] = nsum4r<n>(Yu, i, j, xv[q]);
          wv[q] = (a.zmode == 2) ? __ldcg(W64 + u * pts + k) : 0.0;
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int e = e0 + q * kThreads;
        if (e < cnt) {
          const double x = xv[q];
          double gx;  // g(x) / x
          if (a.zmode == 0) gx = x * x;
          else if (a.zmode == 1) gx = 1.0;
          else if (a.zmode == 2) gx = wv[q] * wv[q];
          else gx = a.wconst;
          z[u * pts + (size_t)a0 * n + e] = fma(x, fma(-dts, gx, m4c1s), c1s * sv[q]);
        }
      }
    }
  }
}

// N2: H = (Y - Yhat) + ih2 lap(z) in FP32; Jacobian weights and their range per item
template <int N>
__device__ __forceinline__ void ph_resid(const PArgs& a, Items its) {
  constexpr int n = N - 1, nb = (n + kDstRows - 1) / kDstRows, U = 4;
  __shared__ float sh[2][kThreads / 32];
  const size_t pts = (size_t)n * n;
  const double* __restrict__ Y = a.Y;
  const double* __restrict__ yhat = a.yhat;
  const double* __restrict__ W64 = a.W64;
  float* __restrict__ rhs = a.rhs;
  float* __restrict__ w = a.w;
  for (int item = its.first; item < its.end; item += its.step) {
    const int u = item / nb, b = item - u * nb, a0 = b * kDstRows;
    if (its.chk && a.flag[2 * u]) continue;
    const double* __restrict__ zu = a.z + u * pts;
    const size_t base = u * pts + (size_t)a0 * n;
    const int cnt = (n - a0 < kDstRows ? n - a0 : kDstRows) * n;
    // range of the FP32 weights: exact in FP32 (min and max round nothing)
    float lo = INFINITY, hi = -INFINITY;
    bool bad = false;  // a non-finite FP64 residual: the state or the step has failed
    for (int e0 = threadIdx.x; e0 < cnt; e0 += U * kThreads) {
      double lz[U], yv[U], hv[U], w64[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int e = e0 + q * kThreads;
        if (e < cnt) {
          const int i = a0 + e / n, j = e - (e / n) * n;
          double zc;
          const double s4 = nsum4r<n>(zu, i, j, zc);  // sets zc (sequenced before its use below)
          lz[q] = s4 - 4.0 * zc;  // h^2 lap(z) of the scaled z: h^-2 folded in
          yv[q] = __ldcg(Y + base + e);
          hv[q] = __ldcg(yhat + base + e);
          w64[q] = (a.zmode == 2) ? __ldcg(W64 + base + e) : 0.0;
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int e = e0 + q * kThreads;
        if (e < cnt) {
          const float hq = float((yv[q] - hv[q]) + lz[q]);
          bad |= !isfinite(hq);
          rhs[base + e] = hq;
          float wq;
          if (a.zmode == 0) {
            const float y = float(yv[q]);
            wq = 3.f * y * y;
          } else if (a.zmode == 1) {
            wq = 1.f;
          } else if (a.zmode == 2) {
            const float y = float(w64[q]);
            wq = y * y;
          } else {
            wq = float(a.wconst);
          }
          w[base + e] = wq;
          lo = fminf(lo, wq);
          hi = fmaxf(hi, wq);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    // (fmin / fmax skip NaN, and a CG started from a non-finite residual can stop at once with a
    // zero correction, so the failure is flagged here)
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, ST_NONFINITE);
    if ((threadIdx.x & 31) == 0) {
      sh[0][threadIdx.x >> 5] = lo;
      sh[1][threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 1; i < kThreads / 32; ++i) {
        lo = fminf(lo, sh[0][i]);
        hi = fmaxf(hi, sh[1][i]);
      }
      a.pmin[(size_t)u * nb + b] = (double)lo;
      a.pmax[(size_t)u * nb + b] = (double)hi;
    }
  }
}

template <int N>
__device__ __forceinline__ void ph_cg_reset(const PArgs& a) {
  for (int u = blockIdx.x * kThreads + threadIdx.x; u < a.units; u += gridDim.x * kThreads) a.flag[2 * u + 1] = 0;
  if (blockIdx.x == 0 && threadIdx.x < 2) a.active[threadIdx.x] = 0;
}

// CG scalars of iteration `it` (Chronopoulos-Gear form: both inner products of an iteration
// come from one reduction, gamma = (r, u) and delta = (w, u) with u = M^{-1} r and w = S u):
//   beta = gamma / gamma_prev (0 at it = 0), alpha = gamma / (delta - beta gamma / alpha_prev).
__device__ __forceinline__ void cg_scalars(int it, double gam, double del, double gp, double ap, double& alpha,
                                           double& beta) {
  beta = 0.0;
  if (it > 0) {
    beta = (gp > 0.0) ? gam / gp : 0.0;
    const double den = (ap != 0.0) ? del - beta * gam / ap : del;
    alpha = (den > 0.0) ? gam / den : 0.0;
  } else {
    alpha = (del > 0.0) ? gam / del : 0.0;
  }
}

// The vector updates of a CG iteration on rows [a0, a0 + kDstRows) of unit u:
//   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = M^{-1} r.
// U: elements per thread whose loads are issued together.
template <int N, int U>
__device__ __forceinline__ void cg_update_rows(const PArgs& a, int u, int a0, int it, float fa, float fb, float cwb,
                                               float fe2dt) {
  constexpr int n = N - 1;
  const size_t pts = (size_t)n * n;
  float* __restrict__ xh = a.xh;
  float* __restrict__ rh = a.rh;
  float* __restrict__ ph = a.ph;
  float* __restrict__ sh = a.sh;
  float* __restrict__ uh = a.uh;
  const float* __restrict__ wh = a.qh;
  const float* __restrict__ mu1 = a.mu1;
  const size_t base = u * pts + (size_t)a0 * n;
  const int cnt = (n - a0 < kDstRows ? n - a0 : kDstRows) * n;
  for (int e0 = threadIdx.x; e0 < cnt; e0 += U * kThreads) {
    float uv[U], wv[U], pv[U], sv[U], xv[U], rv[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int e = e0 + q * kThreads;
      if (e < cnt) {
        uv[q] = __ldcg(uh + base + e);
        wv[q] = __ldcg(wh + base + e);
        pv[q] = (it > 0) ? __ldcg(ph + base + e) : 0.f;
        sv[q] = (it > 0) ? __ldcg(sh + base + e) : 0.f;
        xv[q] = __ldcg(xh + base + e);
        rv[q] = __ldcg(rh + base + e);
      }
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int e = e0 + q * kThreads;
      if (e < cnt) {
        const float mv = mu1[a0 + e / n] + mu1[e - (e / n) * n];
        const float p = uv[q] + fb * pv[q];
        const float sq = wv[q] + fb * sv[q];
        const float r = rv[q] - fa * sq;
        ph[base + e] = p;
        sh[base + e] = sq;
        xh[base + e] = xv[q] + fa * p;
        rh[base + e] = r;
        uh[base + e] = r * __frcp_rn(mdiag(mv, fe2dt, cwb));
      }
    }
  }
}

// The CG update of iteration `it` over the batch; a unit whose gamma has fallen to
// cg_tol^2 gamma_0 is done (its x is kept). The first warp loads the unit's flags, partials,
// wbar and CG history in one round trip, sums the partials with the tree of unit_reduce, and
// thread 0 forms the scalars for the block.
template <int N>
__device__ __forceinline__ void ph_cg_update(const PArgs& a, int it) {
  constexpr int n = N - 1, nb = (n + kDstRows - 1) / kDstRows;
  static_assert(nb <= 32, "one partial per lane");
  const int cur = (it & 1) * 2, prev = ((it + 1) & 1) * 2;
  __shared__ float sab[3];
  __shared__ int sact;
  for (int item = blockIdx.x; item < a.units * nb; item += gridDim.x) {
    const int u = item / nb, b = item - u * nb, a0 = b * kDstRows;
    __syncthreads();  // the previous item's readers of sab / sact are done
    if (threadIdx.x < 32) {
      const int l = threadIdx.x;
      double g = (l < nb) ? __ldcg(a.pgam + (size_t)u * nb + l) : 0.0;
      double d = (l < nb) ? __ldcg(a.pdel + (size_t)u * nb + l) : 0.0;
      int f0 = 0, f1 = 0;
      double wbv = 0.0, g0 = 0.0, gp = 0.0, ap = 0.0;
      if (l == 0) {
        // the CG-done flag of u may be set during this phase by the block of u's first item
        f0 = __ldcg(a.flag + 2 * u);
        f1 = __ldcg(a.flag + 2 * u + 1);
        wbv = __ldcg(a.scal + u * 8 + 4);
        if (it > 0) {
          g0 = __ldcg(a.cgs + u * 8 + 4);
          gp = __ldcg(a.cgs + u * 8 + prev + 1);
          ap = __ldcg(a.cgs + u * 8 + prev);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        g += __shfl_xor_sync(0xffffffffu, g, o);
        d += __shfl_xor_sync(0xffffffffu, d, o);
      }
      if (l == 0) {
        int act = !(f0 || f1);
        double alpha = 0.0, beta = 0.0;
        if (act) {
          const double gam0 = (it == 0) ? g : g0;
          const bool done = !(g > a.cg_tol2 * gam0);  // also catches NaN
          cg_scalars(it, g, d, gp, ap, alpha, beta);
          if (b == 0) {
            atomicAdd(a.totals + 2, 1ull);
            if (done) {
              a.flag[2 * u + 1] = 1;
            } else {
              atomicAdd(a.active + (it & 1), 1);
              a.cgs[u * 8 + cur] = alpha;
              a.cgs[u * 8 + cur + 1] = g;
              if (it == 0) a.cgs[u * 8 + 4] = g;  // gamma_0 (read only for it > 0)
            }
          }
          act = !done;
        }
        sab[0] = float(alpha);
        sab[1] = float(beta);
        sab[2] = a.fdt * float(wbv);
        sact = act;
      }
    }
    __syncthreads();
    if (!sact) continue;
    cg_update_rows<N, 4>(a, u, a0, it, sab[0], sab[1], sab[2], unit_fe2dt(a, u));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.active[(it + 1) & 1] = 0;
    atomicAdd(a.totals, 1ull);
  }
}

// The CG scalars of iteration `it` for every unit still in both loops (the graph execution's loop
// condition): gamma and delta from the unit's item partials (one warp per unit, the shuffle tree
// of unit_reduce), the stop test (a unit whose gamma has fallen to cg_tol^2 gamma_0 is done: flag
// set, x kept), and alpha, beta into cgs. The units are spread over the grid's blocks, a warp per
// unit, so that their FP64 shuffles and divisions run on many SMs' FP64 pipes (in one block they
// queued on one SM's: 14 us per call at 32 units). Each block adds its count of units that go on
// to ctr[2]; the last block to finish (ctr[3]) reads the total, resets both and returns it (-1 in
// every other thread and block).
// The per-unit part of cg_scalars_all for units first, first + step, ... (a warp per unit); adds
// the block's count of units that go on to `going` and of units evaluated to `evaluated`.
template <int N>
__device__ __forceinline__ void cg_scalars_units(const PArgs& a, int it, int first, int step, int& going,
                                                 unsigned long long& evaluated) {
  constexpr int nb = (N - 1 + kDstRows - 1) / kDstRows;
  static_assert(nb <= 32, "one partial per lane");
  const int cur = (it & 1) * 2, prev = ((it + 1) & 1) * 2;
  const int l = threadIdx.x & 31;
  for (int u = first; u < a.units; u += step) {
    if (__ldcg(a.flag + 2 * u) || __ldcg(a.flag + 2 * u + 1)) continue;  // warp-uniform
    double g = (l < nb) ? __ldcg(a.pgam + (size_t)u * nb + l) : 0.0;
    double d = (l < nb) ? __ldcg(a.pdel + (size_t)u * nb + l) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      g += __shfl_xor_sync(0xffffffffu, g, o);
      d += __shfl_xor_sync(0xffffffffu, d, o);
    }
    if (l == 0) {
      double* cg = a.cgs + u * 8;
      const double gam0 = (it == 0) ? g : cg[4];
      double alpha, beta;
      cg_scalars(it, g, d, (it > 0) ? cg[prev + 1] : 0.0, (it > 0) ? cg[prev] : 0.0, alpha, beta);
      atomicAdd(&evaluated, 1ull);
      if (!(g > a.cg_tol2 * gam0)) {  // also catches NaN
        a.flag[2 * u + 1] = 1;
      } else {
        cg[cur] = alpha;
        cg[cur + 1] = g;
        cg[5 + (it & 1)] = beta;
        if (it == 0) cg[4] = g;
        atomicAdd(&going, 1);
      }
    }
  }
}

template <int N>
__device__ __forceinline__ int cg_scalars_all(const PArgs& a, int it) {
  __shared__ int going;
  __shared__ unsigned long long evaluated;
  if (threadIdx.x == 0) {
    going = 0;
    evaluated = 0ull;
  }
  __syncthreads();
  const int wpb = blockDim.x >> 5;
  cg_scalars_units<N>(a, it, blockIdx.x * wpb + (threadIdx.x >> 5), gridDim.x * wpb, going, evaluated);
  __syncthreads();
  int total = -1;
  if (threadIdx.x == 0) {
    atomicAdd(a.totals + 2, evaluated);
    atomicAdd(a.ctr + 2, going);
    __threadfence();  // this block's scalars, flags and count before its arrival
    if (atomicAdd(a.ctr + 3, 1) == (int)gridDim.x - 1) {
      __threadfence();
      total = atomicExch(a.ctr + 2, 0);
      a.ctr[3] = 0;
      atomicAdd(a.totals, 1ull);
    }
  }
  return total;
}

// The vector updates of CG iteration j, with the scalars cg_scalars_all stored, on the rows of
// `item`, if its unit is still in both loops; the block's writes are visible to the block
// afterwards (the transform that follows reads them).
template <int N>
__device__ __forceinline__ void cg_update_item(const PArgs& a, int item, int j) {
  constexpr int nb = (N - 1 + kDstRows - 1) / kDstRows;
  const int u = item / nb, a0 = (item - u * nb) * kDstRows;
  if (a.flag[2 * u] || a.flag[2 * u + 1]) return;  // block-uniform: not written during the phase
  const double* cg = a.cgs + u * 8;
  const float alpha = float(__ldcg(cg + (j & 1) * 2)), beta = float(__ldcg(cg + 5 + (j & 1)));
  cg_update_rows<N, 4>(a, u, a0, j, alpha, beta, a.fdt * float(__ldcg(a.scal + u * 8 + 4)), unit_fe2dt(a, u));
  __syncthreads();
}

// Newton stop test (the tolerance of Section 4.4, read as a bound on the error of the step). The
// increment |d| is below tol; or, from the second increment on, the iteration contracts
// (rho = |d| / |d_prev| < 1/2: the inexact Newton of the CG solves converges linearly at about
// the CG tolerance) and its estimated remaining error rho / (1 - rho) |d| is below tol; or the
// FP64 rounding floor of the residual has been reached (an increment below sqrt(tol) that fails
// to halve the previous one). The error estimate saves the iteration that would only confirm a
// converged step.
__device__ __forceinline__ bool newton_done(double dm, double prev, int m, double tol, double floor_) {
  if (dm <= tol) return true;
  if (m < 2) return false;
  if (dm < 0.5 * prev && dm * dm <= tol * (prev - dm)) return true;
  return dm <= floor_ && dm > 0.5 * prev;
}

// N7: Newton stop test per unit (newton_done)
template <int N>
__device__ __forceinline__ void ph_newton_end(const PArgs& a, int it_n) {
  const int last = (it_n >= a.newton_max - 1);
  for (int u = blockIdx.x * kThreads + threadIdx.x; u < a.units; u += gridDim.x * kThreads) {
    if (a.flag[2 * u]) continue;
    const double dm = unit_max_thread<N>(a.pd, u);
    const int mm = ++a.cnt[u];
    const double prev = a.scal[u * 8 + 6];
    bool done = newton_done(dm, prev, mm, a.tol, a.floor_);
    a.scal[u * 8 + 6] = dm;
    if (!done && last) {
      atomicOr(a.status, ST_NEWTON);
      done = true;
    }
    if (done) {
      a.flag[2 * u] = 1;
      atomicAdd(reinterpret_cast<unsigned long long*>(a.status + 4), (unsigned long long)mm);
      atomicMax(reinterpret_cast<int*>(a.status + 3), mm);
    } else {
      atomicAdd(a.active + 2 + (it_n & 1), 1);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.active[2 + ((it_n + 1) & 1)] = 0;
    atomicAdd(a.totals + 1, 1ull);
  }
}

template <int N, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k2_persist(PArgs args) {
  constexpr int L = 2 * N;
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  float2* twd = smem2 + buf_elems<N>();
  __shared__ PArgs a;
  if (threadIdx.x == 0) a = args;
  for (int m = threadIdx.x; m < L; m += kThreads) twd[m] = args.tw[m];
  __syncthreads();
#define CH_BAR()                                                  \
  if (!grid_barrier(a.bar)) {                                     \
    if (threadIdx.x == 0) atomicOr(a.status, ST_TIMEOUT);         \
    return;                                                       \
  }
  for (int step = 0; step < a.nsteps; ++step) {
    noinl([&] { ph_prologue<N>(a, step); });
    CH_BAR();
    noinl([&] { ph_predict<N>(a, (a.scheme == SCHEME_NL) && (step > 0 || a.have_prev0)); });
    CH_BAR();
    for (int it_n = 0; it_n < a.newton_max; ++it_n) {
      noinl([&] { ph_z<N>(a, grid_items<N>(a)); });
      CH_BAR();
      noinl([&] { ph_resid<N>(a, grid_items<N>(a)); });
      CH_BAR();
      noinl([&] { dst_phase<N, E_PLAIN>(a, buf, twd, a.rhs, a.tmp, 0, nullptr); });  // H to sine space
      CH_BAR();
      noinl([&] { dst_phase<N, E_INIT>(a, buf, twd, a.tmp, nullptr, 0, nullptr); });  // CG start
      noinl([&] { ph_cg_reset<N>(a); });
      CH_BAR();
      for (int it = 0; it < a.cg_max; ++it) {
        noinl([&] { dst_phase<N, E_PLAIN>(a, buf, twd, a.uh, a.tmp, 1, nullptr); });  // u to physical space
        CH_BAR();
        noinl([&] { dst_phase<N, E_WPROD>(a, buf, twd, a.tmp, a.t2, 1, nullptr); });  // dt (wc - wbar) p
        CH_BAR();
        noinl([&] { dst_phase<N, E_PLAIN>(a, buf, twd, a.t2, a.tmp, 1, nullptr); });  // back to sine space
        CH_BAR();
        noinl([&] { dst_phase<N, E_W>(a, buf, twd, a.tmp, nullptr, 1, nullptr); });  // w = S u, (w,u), (r,u)
        CH_BAR();
        noinl([&] { ph_cg_update<N>(a, it); });
        CH_BAR();
        if (*(volatile int*)(a.active + (it & 1)) == 0) break;
      }
      noinl([&] { dst_phase<N, E_PLAIN>(a, buf, twd, a.xh, a.tmp, 0, nullptr); });  // correction to physical space
      CH_BAR();
      noinl([&] { dst_phase<N, E_UPDATE>(a, buf, twd, a.tmp, nullptr, 0, a.pd); });  // Y -= d, max |d|
      CH_BAR();
      noinl([&] { ph_newton_end<N>(a, it_n); });
      CH_BAR();
      if (*(volatile int*)(a.active + 2 + (it_n & 1)) == 0) break;
    }
  }
#undef CH_BAR
}

template <int N, int MINB>
cudaError_t launch_persist(const PArgs& a, int* grid_out, cudaStream_t st) {
  const size_t smem = (size_t)(buf_elems<N>() + 2 * N) * sizeof(float2);
  cudaError_t e = prep(k2_persist<N, MINB>, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2_persist<N, MINB>, kThreads, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  constexpr int nb = (N - 1 + kDstRows - 1) / kDstRows;
  int grid = sms * per_sm;
  if (grid > a.units * nb) grid = a.units * nb;
  *grid_out = grid;
  PArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)k2_persist<N, MINB>, dim3(grid), dim3(kThreads), params, smem, st);
}

// Compiled for two blocks per SM (128 registers per thread): measured fastest at n = 255 among
// 2, 3 and 4.
template <int N>
cudaError_t launch_persist_sel(const PArgs& a, int minb, int* grid_out, cudaStream_t st) {
  (void)minb;
  return launch_persist<N, 2>(a, grid_out, st);
}

// ------------------------------------------------------------------ cluster execution
//
// One thread-block cluster of C blocks per unit runs that unit's whole propagation (nsteps
// implicit steps) in one launch. Block r of a cluster owns the row blocks r, r + C, ... of its
// unit; the phases are the ones above, separated by cluster barriers instead of kernel
// boundaries (barrier.cluster arrive.release / wait.acquire order each phase's global-memory
// writes before the next phase's reads, which are L2-coherent loads), and each unit leaves its
// CG and Newton loops as soon as it has converged instead of when the slowest unit of the batch
// has. Every block of a cluster forms the loop decisions from the same partials summed in the
// same order, so all blocks take the same branches and meet at the same barriers; the loops are
// bounded by cg_max and newton_max.

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ int cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}

__device__ __forceinline__ int cluster_blocks() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return (int)r;
}

__device__ __forceinline__ int cluster_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return (int)r;
}

// Transform passes over this block's items, unit flags not tested (act = -1).
template <int N, int EPI>
__device__ __forceinline__ void dst_items(const PArgs& a, float2* buf, const float2* twd, const float* in, float* out,
                                          double* part, Items its, double wb) {
  for (int item = its.first; item < its.end; item += its.step) {
    __syncthreads();  // the previous item's epilogue has finished reading buf
    noinl([&] { dst_item<N, EPI>(a, buf, twd, in, out, -1, part, item, wb); });
  }
}

template <int N>
__global__ void __launch_bounds__(kThreads, 2) k2_cluster(PArgs args) {
  constexpr int n = N - 1, L = 2 * N, nb = (n + kDstRows - 1) / kDstRows;
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  float2* twd = smem2 + buf_elems<N>();
  __shared__ PArgs a;
  if (threadIdx.x == 0) a = args;
  for (int m = threadIdx.x; m < L; m += kThreads) twd[m] = args.tw[m];
  __syncthreads();
  const int C = cluster_blocks(), rank = cluster_rank(), u = cluster_index();
  if (u >= a.units) return;  // whole clusters only (the grid is units x C blocks)
  const Items its{u * nb + rank, C, (u + 1) * nb, 0};
  long long cg_iters = 0;
  unsigned long long newton_sum = 0;
  int newton_peak = 0;
  unsigned st = 0;
  for (int step = 0; step < a.nsteps; ++step) {
    noinl([&] { ph_prologue_items<N>(a, its); });
    cluster_sync();
    noinl([&] { ph_predict_items<N>(a, (a.scheme == SCHEME_NL) && (step > 0 || a.have_prev0), its); });
    cluster_sync();
    double prev_dm = 0.0;
    int m = 0;
    for (int it_n = 0; it_n < a.newton_max; ++it_n) {
      noinl([&] { ph_z<N>(a, its); });
      cluster_sync();
      noinl([&] { ph_resid<N>(a, its); });
      // the first pass reads only the rows this block has just written
      dst_items<N, E_PLAIN>(a, buf, twd, a.rhs, a.tmp, nullptr, its, 0.0);  // H to sine space
      cluster_sync();
      const double wb = unit_wbar<N>(a, u);
      dst_items<N, E_INIT>(a, buf, twd, a.tmp, nullptr, nullptr, its, wb);  // CG start
      cluster_sync();
      const float cwb = a.fdt * float(wb), fe2dt = unit_fe2dt(a, u);
      double gam0 = 0.0, gp = 0.0, ap = 0.0;
      for (int it = 0; it < a.cg_max; ++it) {
        dst_items<N, E_PLAIN>(a, buf, twd, a.uh, a.tmp, nullptr, its, wb);  // u to physical space
        cluster_sync();
        dst_items<N, E_WPROD>(a, buf, twd, a.tmp, a.t2, nullptr, its, wb);  // dt (wc - wbar) u
        cluster_sync();
        dst_items<N, E_PLAIN>(a, buf, twd, a.t2, a.tmp, nullptr, its, wb);  // back to sine space
        cluster_sync();
        dst_items<N, E_W>(a, buf, twd, a.tmp, nullptr, nullptr, its, wb);  // w = S u, (w,u), (r,u)
        cluster_sync();
        const double gam = unit_reduce<N, 0>(a.pgam, u), del = unit_reduce<N, 0>(a.pdel, u);
        if (it == 0) gam0 = gam;
        ++cg_iters;
        if (!(gam > a.cg_tol2 * gam0)) break;  // also catches NaN
        __shared__ double sab[2];
        if (threadIdx.x == 0) {
          double al, be;
          cg_scalars(it, gam, del, gp, ap, al, be);
          sab[0] = al;
          sab[1] = be;
        }
        __syncthreads();
        const double alpha = sab[0], beta = sab[1];
        gp = gam;
        ap = alpha;
        // the next pass reads only the rows this block updates here
        noinl([&] {
          for (int item = its.first; item < its.end; item += its.step)
            cg_update_rows<N, 8>(a, u, (item - u * nb) * kDstRows, it, float(alpha), float(beta), cwb, fe2dt);
        });
      }
      dst_items<N, E_PLAIN>(a, buf, twd, a.xh, a.tmp, nullptr, its, 0.0);  // correction to physical space
      cluster_sync();
      dst_items<N, E_UPDATE>(a, buf, twd, a.tmp, nullptr, a.pd, its, 0.0);  // Y -= d, max |d|
      cluster_sync();
      const double dm = unit_reduce<N, 1>(a.pd, u);
      ++m;
      bool done = newton_done(dm, prev_dm, m, a.tol, a.floor_);
      prev_dm = dm;
      if (!done && it_n == a.newton_max - 1) {
        st |= ST_NEWTON;
        done = true;
      }
      if (done) break;
    }
    newton_sum += (unsigned long long)m;
    newton_peak = m > newton_peak ? m : newton_peak;
  }
  if (rank == 0 && threadIdx.x == 0) {
    if (st) atomicOr(a.status, st);
    atomicAdd(reinterpret_cast<unsigned long long*>(a.status + 4), newton_sum);
    atomicMax(reinterpret_cast<int*>(a.status + 3), newton_peak);
    atomicAdd(a.totals + 2, (unsigned long long)cg_iters);
  }
}

template <int N>
cudaError_t cluster_prepare() {
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(dev)) return cudaSuccess;
  e = cudaFuncSetAttribute(k2_cluster<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dst_smem<N>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_cluster<N>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) done.insert(dev);
  return e;
}

template <int N>
void cluster_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* at, int units, int C, cudaStream_t st) {
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3((unsigned)(units * C));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = dst_smem<N>();
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
}

// Cluster size for `units` units: the largest power of two up to min(16, row blocks) for which
// all clusters are resident at once, else 1 (one block per unit, in waves). `force` > 0 takes
// that size if it divides the row blocks.
template <int N>
cudaError_t cluster_choose(int units, int force, int* C_out) {
  constexpr int nb = (N - 1 + kDstRows - 1) / kDstRows;
  cudaError_t e = cluster_prepare<N>();
  if (e != cudaSuccess) return e;
  if (force > 0 && force <= 16 && nb % force == 0) {
    *C_out = force;
    return cudaSuccess;
  }
  for (int C = nb < 16 ? nb : 16; C > 1; C /= 2) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    cluster_config<N>(cfg, at, units, C, nullptr);
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, k2_cluster<N>, &cfg);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      continue;
    }
    if (ncl >= units) {
      *C_out = C;
      return cudaSuccess;
    }
  }
  *C_out = 1;
  return cudaSuccess;
}

template <int N>
cudaError_t launch_cluster(const PArgs& a, int force, int* C_out, cudaStream_t st) {
  int C = 1;
  cudaError_t e = cluster_choose<N>(a.units, force, &C);
  if (e != cudaSuccess) return e;
  *C_out = C;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  cluster_config<N>(cfg, at, a.units, C, st);
  return cudaLaunchKernelEx(&cfg, k2_cluster<N>, a);
}

}  // namespace

void Prop2D::make_args(PArgs& a, double* Y, int units, int scheme, double dt, int nsteps, int u0, int group) const {
  a = PArgs{};
  const int nb = (p_.n + kDstRows - 1) / kDstRows;
  const size_t np = (size_t)cap_ * nb;
  const size_t vo = (size_t)u0 * pts_, po = (size_t)u0 * nb;  // offsets of unit u0
  a.Y = Y;
  a.yhat = yhat_ + vo;
  a.yprev = yprev_ + vo;
  a.z = z_ + vo;
  a.w = w_ + vo;
  a.rhs = rhs_ + vo;
  a.xh = xh_ + vo;
  a.rh = rh_ + vo;
  a.ph = ph_ + vo;
  a.qh = qh_ + vo;
  a.tmp = tmp_ + vo;
  a.t2 = tmp2_ + vo;
  a.mu1 = mu_;
  a.tw = tw_;
  a.pmin = ppart_ + po;
  a.pmax = ppart_ + np + po;
  a.pdel = ppart_ + 2 * np + po;
  a.pgam = ppart_ + 3 * np + po;
  a.cgs = cgs_ + (size_t)u0 * 8;
  a.uh = uh_ + vo;
  a.sh = sh_ + vo;
  a.pd = ppart_ + 6 * np + po;
  a.flag = flag_ + (size_t)u0 * 2;
  a.cnt = newton_cnt_ + u0;
  a.scal = scal_ + (size_t)u0 * 8;
  a.status = status_;
  a.totals = cg_dev_;
  a.active = active_ + 4 * group;
  a.bar = bar_;
  a.units = units;
  a.nsteps = nsteps;
  a.scheme = scheme;
  a.newton_max = p_.newton_max;
  a.cg_max = p_.cg_max;
  a.have_prev0 = 0;
  a.frozen = p_.frozen;
  a.dt = dt;
  a.ih2 = 1.0 / (p_.h * p_.h);
  a.c1 = p_.eps2 * dt * a.ih2;
  a.tol = p_.newton_tol;
  a.floor_ = std::sqrt(p_.newton_tol);
  a.cg_tol2 = p_.cg_tol * p_.cg_tol;
  a.fe2dt = float(p_.eps2 * dt);
  a.eps2 = p_.eps2;
  a.eps2u = eps2u_ ? eps2u_ + u0 : nullptr;
  a.fdt = float(dt);
  if (scheme == SCHEME_NL) {
    a.zmode = p_.frozen ? 1 : 0;
  } else if (scheme == SCHEME_LIN1) {
    a.zmode = p_.frozen ? 3 : 2;
    a.W64 = yprev_ + vo;
    a.wconst = 1.0;
  } else {
    a.zmode = 3;
    a.wconst = 2.0;
  }
  a.ctr = ctr_ + 4 * group;
}

cudaError_t Prop2D::propagate_persistent(double* Y, int units, int scheme, double dt, int nsteps, cudaStream_t st) {
  if (units > cap_ || units < 1) return cudaErrorInvalidValue;
  if (nsteps < 1) return cudaSuccess;
  PArgs a;
  make_args(a, Y, units, scheme, dt, nsteps, 0, 0);
  cudaError_t e = cudaMemsetAsync(bar_, 0, 4 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  int grid = 0;
  const int minb = persist_minb_;
  switch (p_.n + 1) {
    case 16: e = launch_persist_sel<16>(a, minb, &grid, st); break;
    case 32: e = launch_persist_sel<32>(a, minb, &grid, st); break;
    case 64: e = launch_persist_sel<64>(a, minb, &grid, st); break;
    case 128: e = launch_persist_sel<128>(a, minb, &grid, st); break;
    case 256: e = launch_persist_sel<256>(a, minb, &grid, st); break;
    case 512: e = launch_persist_sel<512>(a, minb, &grid, st); break;
    default: e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) step_kernels_ += 1;
  return e;
}


cudaError_t Prop2D::propagate_cluster(double* Y, int units, int scheme, double dt, int nsteps, cudaStream_t st) {
  if (units > cap_ || units < 1) return cudaErrorInvalidValue;
  if (nsteps < 1) return cudaSuccess;
  PArgs a;
  make_args(a, Y, units, scheme, dt, nsteps, 0, 0);
  a.have_prev0 = 0;
  cudaError_t e = cudaSuccess;
  int C = 1;
  switch (p_.n + 1) {
    case 16: e = launch_cluster<16>(a, cluster_force_, &C, st); break;
    case 32: e = launch_cluster<32>(a, cluster_force_, &C, st); break;
    case 64: e = launch_cluster<64>(a, cluster_force_, &C, st); break;
    case 128: e = launch_cluster<128>(a, cluster_force_, &C, st); break;
    case 256: e = launch_cluster<256>(a, cluster_force_, &C, st); break;
    case 512: e = launch_cluster<512>(a, cluster_force_, &C, st); break;
    default: e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) {
    step_kernels_ += 1;
    cluster_size_ = C;
  }
  return e;
}

// ------------------------------------------------------------------ graph execution
//
// The same phases as separate kernels (each at its own occupancy), one CUDA graph per step with
// the Newton and CG loops as conditional WHILE nodes. Loop indices live in device counters
// (ctr[0] Newton, ctr[1] CG), advanced by the condition kernels.
namespace {

// PH_P1U: the CG update of the previous iteration on the item's rows, then P1 on them;
// PH_X1U: the update of the last iteration for units that left the CG loop at cg_max, then X1.
// PH_P4S: P4, then the last block to finish forms the CG scalars of every unit and sets the CG
// loop's condition (small batches: no separate scalar kernel).
enum Phase {
  PH_PROLOGUE = 0, PH_PREDICT, PH_Z, PH_RESID, PH_H1, PH_H2, PH_P1, PH_P2, PH_P3, PH_P4, PH_UPDATE,
  PH_X1, PH_X2, PH_NEWTON_END, PH_P1U, PH_X1U, PH_P4S
};

__host__ __device__ constexpr bool is_dst_phase(int ph) {
  return ph == PH_H1 || ph == PH_H2 || ph == PH_P1 || ph == PH_P2 || ph == PH_P3 || ph == PH_P4 || ph == PH_X1 ||
         ph == PH_X2 || ph == PH_P1U || ph == PH_X1U || ph == PH_P4S;
}

// Batches of at most this many units end a CG iteration with PH_P4S instead of P4 and the scalar
// kernel: one launch fewer per CG iteration where the scalar work is a few warps' worth.
constexpr int kFuseScalarUnits = 4;

// Four blocks per SM: 64 registers hold the 16 complex values a lane carries through the warp
// FFTs of 256 x 256 and 512 x 512 (at 256 x 256 a batch's items are then all resident).
template <int N, int PH>
__global__ void __launch_bounds__(kThreads, 4) k2_phase(PArgs a, int have_prev) {
  constexpr int L = 2 * N, nb = (N - 1 + kDstRows - 1) / kDstRows;
  extern __shared__ float2 smem2[];
  float2* buf = smem2;
  float2* twd = smem2 + buf_elems<N>();
  if constexpr (is_dst_phase(PH)) {
    for (int m = threadIdx.x; m < L; m += kThreads) twd[m] = a.tw[m];
    __syncthreads();
  }
  const int it = a.ctr[1];
  (void)nb;
  if constexpr (PH == PH_PROLOGUE) ph_prologue<N>(a, 0);
  if constexpr (PH == PH_PREDICT) ph_predict<N>(a, have_prev);
  if constexpr (PH == PH_Z) ph_z<N>(a, grid_items<N>(a));
  if constexpr (PH == PH_RESID) ph_resid<N>(a, grid_items<N>(a));
  if constexpr (PH == PH_H1) dst_item<N, E_PLAIN>(a, buf, twd, a.rhs, a.tmp, 0, nullptr, blockIdx.x);
  if constexpr (PH == PH_H2) {
    dst_item<N, E_INIT>(a, buf, twd, a.tmp, nullptr, 0, nullptr, blockIdx.x);
    ph_cg_reset<N>(a);
  }
  if constexpr (PH == PH_P1) dst_item<N, E_PLAIN>(a, buf, twd, a.uh, a.tmp, 1, nullptr, blockIdx.x);
  if constexpr (PH == PH_P2) dst_item<N, E_WPROD>(a, buf, twd, a.tmp, a.t2, 1, nullptr, blockIdx.x);
  if constexpr (PH == PH_P3) dst_item<N, E_PLAIN>(a, buf, twd, a.t2, a.tmp, 1, nullptr, blockIdx.x);
  if constexpr (PH == PH_P4) dst_item<N, E_W>(a, buf, twd, a.tmp, nullptr, 1, nullptr, blockIdx.x);
  if constexpr (PH == PH_P4S) {
    dst_item<N, E_W>(a, buf, twd, a.tmp, nullptr, 1, nullptr, blockIdx.x);
    __shared__ int last, going;
    __shared__ unsigned long long evaluated;
    __syncthreads();  // the block's partials are written (or its unit is done)
    if (threadIdx.x == 0) {
      __threadfence();
      last = (atomicAdd(a.ctr + 3, 1) == (int)gridDim.x - 1);
      going = 0;
      evaluated = 0ull;
    }
    __syncthreads();
    if (last) {
      __threadfence();  // every block's partials before they are summed
      cg_scalars_units<N>(a, it, threadIdx.x >> 5, kThreads >> 5, going, evaluated);
      __syncthreads();
      if (threadIdx.x == 0) {
        a.ctr[3] = 0;
        atomicAdd(a.totals + 2, evaluated);
        atomicAdd(a.totals, 1ull);
        a.ctr[1] = it + 1;
        cudaGraphSetConditional(a.hcg, (going > 0 && it + 1 < a.cg_max) ? 1u : 0u);
      }
    }
  }

  if constexpr (PH == PH_UPDATE) ph_cg_update<N>(a, it);
  if constexpr (PH == PH_X1) dst_item<N, E_PLAIN>(a, buf, twd, a.xh, a.tmp, 0, nullptr, blockIdx.x);
  if constexpr (PH == PH_P1U) {
    if (it > 0) cg_update_item<N>(a, blockIdx.x, it - 1);
    dst_item<N, E_PLAIN>(a, buf, twd, a.uh, a.tmp, 1, nullptr, blockIdx.x);
  }
  if constexpr (PH == PH_X1U) {
    if (it > 0) cg_update_item<N>(a, blockIdx.x, it - 1);  // it = CG iterations run
    dst_item<N, E_PLAIN>(a, buf, twd, a.xh, a.tmp, 0, nullptr, blockIdx.x);
  }
  if constexpr (PH == PH_X2) dst_item<N, E_UPDATE>(a, buf, twd, a.tmp, nullptr, 0, a.pd, blockIdx.x);
  if constexpr (PH == PH_NEWTON_END) ph_newton_end<N>(a, a.ctr[0]);
}

// End of a loop iteration: continue while units remain active and the cap is not reached.
// which = 0: Newton (active slots 2, 3), 1: CG (slots 0, 1).
// End of a CG iteration of the graph execution: the scalars of every unit (cg_scalars_all), then
// (in the last block to finish) continue while units go on and the cap is not reached. Blocks of
// kScalarThreads, a warp per unit: scalar_blocks(units) of them.
constexpr int kScalarThreads = 64;
inline int scalar_blocks(int units) {
  const int b = (units + kScalarThreads / 32 - 1) / (kScalarThreads / 32);
  return b < 1 ? 1 : (b > 1024 ? 1024 : b);
}

template <int N>
__global__ void __launch_bounds__(kScalarThreads) k2_cg_cond(PArgs a, cudaGraphConditionalHandle hnd, int lim) {
  const int it = a.ctr[1];
  const int going = cg_scalars_all<N>(a, it);
  if (going >= 0) {  // the last block's thread 0: every block has read ctr[1]
    a.ctr[1] = it + 1;
    cudaGraphSetConditional(hnd, (going > 0 && it + 1 < lim) ? 1u : 0u);
  }
}

// The same for the host-driven execution: the count goes to active[it & 1] for the host.
template <int N>
__global__ void __launch_bounds__(kScalarThreads) k2_cg_host(PArgs a) {
  const int it = a.ctr[1];
  const int going = cg_scalars_all<N>(a, it);
  if (going >= 0) a.active[it & 1] = going;
}

__global__ void k2_cond(cudaGraphConditionalHandle hnd, int* __restrict__ ctr, const int* __restrict__ active,
                        int which, int lim) {
  if (threadIdx.x == 0) {
    const int it = ctr[which];
    const int c = active[(which == 0 ? 2 : 0) + (it & 1)];
    ctr[which] = it + 1;
    cudaGraphSetConditional(hnd, (c > 0 && it + 1 < lim) ? 1u : 0u);
  }
}

template <int N, int PH>
cudaError_t phase_launch(const PArgs& a, int have_prev, cudaStream_t st) {
  constexpr int nb = (N - 1 + kDstRows - 1) / kDstRows;
  const size_t smem = is_dst_phase(PH) ? (size_t)(buf_elems<N>() + 2 * N) * sizeof(float2) : 0;
  k2_phase<N, PH><<<a.units * nb, kThreads, smem, st>>>(a, have_prev);
  return cudaGetLastError();
}

template <int N>
cudaError_t phase_prepare() {
  const size_t smem = (size_t)(buf_elems<N>() + 2 * N) * sizeof(float2);
  cudaError_t e = prep(k2_phase<N, PH_H1>, smem);
  if (e == cudaSuccess) e = prep(k2_phase<N, PH_H2>, smem);
  if (e == cudaSuccess) e = prep(k2_phase<N, PH_P1>, smem);
  if (e == cudaSuccess) e = prep(k2_phase<N, PH_P2>, smem);
  if (e == cudaSuccess) e = prep(k2_phase<N, PH_P3>, smem);
  if (e == cudaSuccess) e = prep(k2_phase<N, PH_P4>, smem);
  if (e == cudaSuccess) e = prep(k2_phase<N, PH_X1>, smem);
  if (e == cudaSuccess) e = prep(k2_phase<N, PH_X2>, smem);
  if (e == cudaSuccess) e = prep(k2_phase<N, PH_P1U>, smem);
  if (e == cudaSuccess) e = prep(k2_phase<N, PH_X1U>, smem);
  if (e == cudaSuccess) e = prep(k2_phase<N, PH_P4S>, smem);
  return e;
}

// The step graph of one grid size.
template <int N>
cudaError_t build_step_n(const PArgs& a, int have_prev, int newton_max, int cg_max, int* ctr, int* active,
                         cudaGraphExec_t* out) {
  cudaError_t e = phase_prepare<N>();
  if (e != cudaSuccess) return e;
  cudaStream_t cs = nullptr, bs = nullptr, bs2 = nullptr;
  cudaGraph_t g = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  cudaGraphConditionalHandle hN = 0, hC = 0;
  if (e == cudaSuccess) e = phase_launch<N, PH_PROLOGUE>(a, have_prev, cs);
  if (e == cudaSuccess) e = phase_launch<N, PH_PREDICT>(a, have_prev, cs);
  if (e == cudaSuccess) e = capture_graph(cs, &g);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hN, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    k2_loop_start<<<1, 32, 0, cs>>>(hN, ctr, 0, 0);
    e = cudaGetLastError();
  }
  cudaGraph_t bodyN = nullptr;
  if (e == cudaSuccess) e = add_while(cs, &hN, 1, cudaGraphCondAssignDefault, &bodyN);
  // ---- Newton body
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(bs, bodyN, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = phase_launch<N, PH_Z>(a, have_prev, bs);
  if (e == cudaSuccess) e = phase_launch<N, PH_RESID>(a, have_prev, bs);
  if (e == cudaSuccess) e = phase_launch<N, PH_H1>(a, have_prev, bs);
  if (e == cudaSuccess) e = phase_launch<N, PH_H2>(a, have_prev, bs);
  cudaGraph_t gN = nullptr;
  if (e == cudaSuccess) e = capture_graph(bs, &gN);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hC, gN, 0, 0);
  if (e == cudaSuccess) {
    k2_loop_start<<<1, 32, 0, bs>>>(hC, ctr, 1, 1);
    e = cudaGetLastError();
  }
  cudaGraph_t bodyC = nullptr;
  if (e == cudaSuccess) e = add_while(bs, &hC, 0, 0, &bodyC);
  // ---- CG body
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(bs2, bodyC, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = phase_launch<N, PH_P1U>(a, have_prev, bs2);
  if (e == cudaSuccess) e = phase_launch<N, PH_P2>(a, have_prev, bs2);
  if (e == cudaSuccess) e = phase_launch<N, PH_P3>(a, have_prev, bs2);
  if (a.units <= kFuseScalarUnits) {
    PArgs a4 = a;
    a4.hcg = hC;
    a4.cg_max = cg_max;
    if (e == cudaSuccess) e = phase_launch<N, PH_P4S>(a4, have_prev, bs2);
  } else {
    if (e == cudaSuccess) e = phase_launch<N, PH_P4>(a, have_prev, bs2);
    if (e == cudaSuccess) {
      k2_cg_cond<N><<<scalar_blocks(a.units), kScalarThreads, 0, bs2>>>(a, hC, cg_max);
      e = cudaGetLastError();
    }
  }
  {
    cudaGraph_t dummy = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(bs2, &dummy);
    if (e == cudaSuccess) e = e2;
  }
  // ---- back in the Newton body: last CG update, correction to physical space, update, stop test
  if (e == cudaSuccess) e = phase_launch<N, PH_X1U>(a, have_prev, bs);
  if (e == cudaSuccess) e = phase_launch<N, PH_X2>(a, have_prev, bs);
  if (e == cudaSuccess) e = phase_launch<N, PH_NEWTON_END>(a, have_prev, bs);
  if (e == cudaSuccess) {
    k2_cond<<<1, 32, 0, bs>>>(hN, ctr, active, 0, newton_max);
    e = cudaGetLastError();
  }
  {
    cudaGraph_t dummy = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(bs, &dummy);
    if (e == cudaSuccess) e = e2;
  }
  {
    cudaGraph_t dummy = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &dummy);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  if (bs) cudaStreamDestroy(bs);
  if (bs2) cudaStreamDestroy(bs2);
  return e;
}

}  // namespace

cudaError_t Prop2D::build_step(const StepKey& k, cudaGraphExec_t* out) {
  PArgs a;
  make_args(a, k.Y, k.units, k.scheme, k.dt, 1, k.u0, k.group);
  switch (p_.n + 1) {
    case 16: return build_step_n<16>(a, k.have_prev, p_.newton_max, p_.cg_max, a.ctr, a.active, out);
    case 32: return build_step_n<32>(a, k.have_prev, p_.newton_max, p_.cg_max, a.ctr, a.active, out);
    case 64: return build_step_n<64>(a, k.have_prev, p_.newton_max, p_.cg_max, a.ctr, a.active, out);
    case 128: return build_step_n<128>(a, k.have_prev, p_.newton_max, p_.cg_max, a.ctr, a.active, out);
    case 256: return build_step_n<256>(a, k.have_prev, p_.newton_max, p_.cg_max, a.ctr, a.active, out);
    case 512: return build_step_n<512>(a, k.have_prev, p_.newton_max, p_.cg_max, a.ctr, a.active, out);
  }
  return cudaErrorInvalidValue;
}


// Host-driven execution of the same phases (plain launches; the loop conditions are read back
// after each iteration). Slower than the graphs, but every kernel is an ordinary launch, which
// profilers can attribute one by one (they cannot inside graphs with conditional nodes).
namespace {

template <int N>
cudaError_t host_step_n(const PArgs& a, int have_prev, int newton_max, int cg_max, int* ctr, int* active,
                        int* host_buf, cudaStream_t st) {
  cudaError_t e = phase_prepare<N>();
  if (e != cudaSuccess) return e;
  int* hc = host_buf;      // [0..1] loop counters
  int* act = host_buf + 2; // [0..3] active counts
#define CH_TRY(x)                             \
  do {                                        \
    if ((e = (x)) != cudaSuccess) return e;   \
  } while (0)
  CH_TRY((phase_launch<N, PH_PROLOGUE>(a, have_prev, st)));
  CH_TRY((phase_launch<N, PH_PREDICT>(a, have_prev, st)));
  for (int itn = 0; itn < newton_max; ++itn) {
    hc[0] = itn;
    hc[1] = 0;
    CH_TRY(cudaMemcpyAsync(ctr, hc, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
    CH_TRY((phase_launch<N, PH_Z>(a, have_prev, st)));
    CH_TRY((phase_launch<N, PH_RESID>(a, have_prev, st)));
    CH_TRY((phase_launch<N, PH_H1>(a, have_prev, st)));
    CH_TRY((phase_launch<N, PH_H2>(a, have_prev, st)));
    int ran = 0;
    for (int it = 0; it < cg_max; ++it) {
      hc[1] = it;
      CH_TRY(cudaMemcpyAsync(ctr, hc, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
      CH_TRY((phase_launch<N, PH_P1U>(a, have_prev, st)));
      CH_TRY((phase_launch<N, PH_P2>(a, have_prev, st)));
      CH_TRY((phase_launch<N, PH_P3>(a, have_prev, st)));
      CH_TRY((phase_launch<N, PH_P4>(a, have_prev, st)));
      k2_cg_host<N><<<scalar_blocks(a.units), kScalarThreads, 0, st>>>(a);
      CH_TRY(cudaGetLastError());
      CH_TRY(cudaMemcpyAsync(act, active, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
      CH_TRY(cudaStreamSynchronize(st));
      ++ran;
      if (act[it & 1] == 0) break;
    }
    hc[1] = ran;  // CG iterations run: the last one's update is applied with the correction pass
    CH_TRY(cudaMemcpyAsync(ctr, hc, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
    CH_TRY((phase_launch<N, PH_X1U>(a, have_prev, st)));
    CH_TRY((phase_launch<N, PH_X2>(a, have_prev, st)));
    CH_TRY((phase_launch<N, PH_NEWTON_END>(a, have_prev, st)));
    CH_TRY(cudaMemcpyAsync(act, active, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CH_TRY(cudaStreamSynchronize(st));
    if (act[2 + (itn & 1)] == 0) break;
  }
#undef CH_TRY
  return cudaSuccess;
}

}  // namespace

cudaError_t Prop2D::propagate_host(double* Y, int units, int scheme, double dt, int nsteps, cudaStream_t st) {
  for (int j = 0; j < nsteps; ++j) {
    PArgs a;
    make_args(a, Y, units, scheme, dt, 1, 0, 0);
    const int hp = (scheme == SCHEME_NL && j > 0) ? 1 : 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (p_.n + 1) {
      case 16: e = host_step_n<16>(a, hp, p_.newton_max, p_.cg_max, ctr_, active_, host_cnt_, st); break;
      case 32: e = host_step_n<32>(a, hp, p_.newton_max, p_.cg_max, ctr_, active_, host_cnt_, st); break;
      case 64: e = host_step_n<64>(a, hp, p_.newton_max, p_.cg_max, ctr_, active_, host_cnt_, st); break;
      case 128: e = host_step_n<128>(a, hp, p_.newton_max, p_.cg_max, ctr_, active_, host_cnt_, st); break;
      case 256: e = host_step_n<256>(a, hp, p_.newton_max, p_.cg_max, ctr_, active_, host_cnt_, st); break;
      case 512: e = host_step_n<512>(a, hp, p_.newton_max, p_.cg_max, ctr_, active_, host_cnt_, st); break;
    }
    if (e != cudaSuccess) return e;
    step_kernels_ += 2;  // prologue, predictor
  }
  return cudaSuccess;
}

}  // namespace chg2
