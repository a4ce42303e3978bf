// Learned coarse propagator G_theta(U) = U + R(U) on sm_103a: inference and training kernels.
//
// R is six 3x3 convolutions with zero padding (u = 0 outside the interior grid, Section 2.1),
// channels 1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU after the first five. Activations are BF16,
// channels last ([B][S][S][32]); accumulation is FP32.
//
// The four 32 -> 32 layers carry almost all of the arithmetic (2 x 32 x 288 flops per pixel each)
// and run as an implicit GEMM on the tensor cores: M = 16 output pixels of a row, N = 8 output
// channels, K = 16 input channels of one tap, 18 K-steps (9 taps x 2 channel halves) per tile,
// mma.sync m16n8k16 BF16 x BF16 -> FP32. A CTA computes a 16 x 16 pixel tile from an 18 x 18 halo
// tile in shared memory (pixel stride 80 B so the eight ldmatrix rows of a phase fall on
// distinct banks). The backward pass through a 32 -> 32 layer is the same kernel with taps
// flipped and channels swapped, its epilogue multiplying by the ReLU mask of the layer below.
// The 1 -> 32 and 32 -> 1 layers, the weight gradients (per-tile partials reduced in a fixed
// order), the loss and Adam (Kingma and Ba, 2015) run on the CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "ch_ctx.cuh"
#include "ch_trace.cuh"
#include "ch_wait.cuh"
#include "gtheta.cuh"

namespace chg3 {

namespace {

using bf16 = __nv_bfloat16;
constexpr int kTile = 16;        // output tile edge
constexpr int kHalo = kTile + 2;
constexpr int kPix = 40;         // BF16 elements per pixel in shared tiles (80 B)
constexpr int kThreads = 256;
// scalar copies of the layout offsets for device code
constexpr int kW1 = kOffW[0], kW2 = kOffW[1], kW6 = kOffW[5], kMidStride = kOffW[2] - kOffW[1];
static_assert(kOffW[3] - kOffW[2] == kMidStride && kOffW[4] - kOffW[3] == kMidStride, "layout");
static_assert(kOffB[0] == kW1 + 9 * kC && kOffB[5] == kW6 + 9 * kC, "layout");

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}

__device__ __forceinline__ void mma16816(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros (the halo outside the
// field).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Issues the asynchronous loads of the 18 x 18 halo tile at (ty0, tx0) of a [S][S][32] field.
__device__ __forceinline__ void load_halo_async(bf16* tile, const bf16* __restrict__ x, int S, int ty0, int tx0) {
  for (int c = threadIdx.x; c < kHalo * kHalo * 4; c += kThreads) {
    const int pix = c >> 2, part = c & 3;
    const int yy = pix / kHalo, xx = pix - yy * kHalo;
    const int gy = ty0 - 1 + yy, gx = tx0 - 1 + xx;
    const bool in = gy >= 0 && gy < S && gx >= 0 && gx < S;
    const bf16* src = in ? x + ((size_t)gy * S + gx) * kC + part * 8 : x;
    cp_async16(tile + pix * kPix + part * 8, src, in ? 16 : 0);
  }
}

// Loads the 18 x 18 halo tile of a [S][S][32] BF16 field into shared memory (zeros outside).
__device__ __forceinline__ void load_halo(bf16* tile, const bf16* __restrict__ x, int S, int ty0, int tx0) {
  for (int c = threadIdx.x; c < kHalo * kHalo * 4; c += kThreads) {
    const int pix = c >> 2, part = c & 3;
    const int yy = pix / kHalo, xx = pix - yy * kHalo;
    const int gy = ty0 - 1 + yy, gx = tx0 - 1 + xx;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gy >= 0 && gy < S && gx >= 0 && gx < S)
      v = *reinterpret_cast<const uint4*>(x + ((size_t)gy * S + gx) * kC + part * 8);
    *reinterpret_cast<uint4*>(tile + pix * kPix + part * 8) = v;
  }
}

// 32 -> 32 convolution on the tensor cores, persistent over 16 x 16 output tiles: a CTA loads the
// layer's weights into shared memory once and walks tiles (t = blockIdx.x, + gridDim.x, ...;
// tile t = (image, tile row, tile column)); the halo of the next tile is fetched with cp.async
// into the second of two buffers while the current one is multiplied.
// mode 0 (forward): y = relu(conv(x, W) + b); mode 1 (backward data): y = conv(x, W) * (mask > 0).
constexpr int kHaloElems = kHalo * kHalo * kPix;
constexpr size_t kConvSmem = (2 * kHaloElems + 9 * kC * kPix) * sizeof(bf16);

__global__ void __launch_bounds__(kThreads, 2) k_conv_mid(const bf16* __restrict__ x, bf16* __restrict__ y,
                                                          const bf16* __restrict__ W, const float* __restrict__ bias,
                                                          const bf16* __restrict__ mask, int S, int tiles_x,
                                                          int tiles, int mode) {
  extern __shared__ __align__(16) unsigned char conv_smem[];
  bf16* halo = reinterpret_cast<bf16*>(conv_smem);  // two buffers
  bf16* ws = halo + 2 * kHaloElems;
  const int per_img = tiles_x * tiles_x;
  auto tile_origin = [&](int tl, int& img, int& ty0, int& tx0) {
    img = tl / per_img;
    const int r = tl - img * per_img;
    ty0 = (r / tiles_x) * kTile;
    tx0 = (r % tiles_x) * kTile;
  };
  if (blockIdx.x < tiles) {
    int img, ty0, tx0;
    tile_origin(blockIdx.x, img, ty0, tx0);
    load_halo_async(halo, x + (size_t)img * S * S * kC, S, ty0, tx0);
  }
  cp_async_commit();
  for (int c = threadIdx.x; c < 9 * kC * 4; c += kThreads) {
    const int row = c >> 2, part = c & 3;  // row = tap * 32 + output channel
    *reinterpret_cast<uint4*>(ws + row * kPix + part * 8) = *reinterpret_cast<const uint4*>(W + row * kC + part * 8);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int arow = (lane & 7) + ((lane >> 3) & 1) * 8;
  const int akof = (lane >> 4) * 8;
  float bv[4][2];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    bv[j][0] = (mode == 0) ? bias[j * 8 + 2 * t] : 0.f;
    bv[j][1] = (mode == 0) ? bias[j * 8 + 2 * t + 1] : 0.f;
  }
  int buf = 0;
  for (int tl = blockIdx.x; tl < tiles; tl += gridDim.x, buf ^= 1) {
    int img, ty0, tx0;
    tile_origin(tl, img, ty0, tx0);
    const size_t off = (size_t)img * S * S * kC;
    const int nxt = tl + gridDim.x;
    if (nxt < tiles) {  // the other buffer was released by the barrier closing the previous tile
      int im2, y2, x2;
      tile_origin(nxt, im2, y2, x2);
      load_halo_async(halo + (buf ^ 1) * kHaloElems, x + (size_t)im2 * S * S * kC, S, y2, x2);
    }
    cp_async_commit();
    cp_async_wait<1>();  // this tile's group has landed (the next one may still be in flight)
    __syncthreads();
    const bf16* tile = halo + buf * kHaloElems;
    float acc[2][4][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][j][q] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3, dx = tap - 3 * dy;
#pragma unroll
      for (int kh = 0; kh < 2; ++kh) {
        const int c0 = kh * 16;
        unsigned a[2][4];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          const int oy = warp * 2 + m;
          ldsm_x4(a[m][0], a[m][1], a[m][2], a[m][3], tile + ((oy + dy) * kHalo + arow + dx) * kPix + c0 + akof);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bf16* wb = ws + (tap * kC + j * 8 + g) * kPix + c0 + 2 * t;
          const unsigned b0 = *reinterpret_cast<const unsigned*>(wb);
          const unsigned b1 = *reinterpret_cast<const unsigned*>(wb + 8);
#pragma unroll
          for (int m = 0; m < 2; ++m) mma16816(acc[m][j], a[m], b0, b1);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int Y = ty0 + warp * 2 + m;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int co = j * 8 + 2 * t;
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int X = tx0 + g + 8 * hf;
          if (Y >= S || X >= S) continue;
          const size_t o = off + ((size_t)Y * S + X) * kC + co;
          float v0 = acc[m][j][2 * hf], v1 = acc[m][j][2 * hf + 1];
          if (mode == 0) {
            v0 = fmaxf(v0 + bv[j][0], 0.f);
            v1 = fmaxf(v1 + bv[j][1], 0.f);
          } else {
            const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(mask + o);
            v0 = (__bfloat162float(mk.x) > 0.f) ? v0 : 0.f;
            v1 = (__bfloat162float(mk.y) > 0.f) ? v1 : 0.f;
          }
          *reinterpret_cast<__nv_bfloat162*>(y + o) = __floats2bfloat162_rn(v0, v1);
        }
      }
    }
    __syncthreads();  // every warp is done with this buffer before the next prefetch reuses it
  }
  cp_async_wait<0>();
}


// ---------------------------------------------------------------- tcgen05 (5th-generation) path
//
// The same 32 -> 32 convolution issued as tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, one CTA)
// with the accumulators in tensor memory. Operands are read by the tensor core through shared-
// memory matrix descriptors in the K-major layout without swizzle: a core matrix is 8 rows of
// 16 bytes (8 channels), consecutive in memory; LBO is the distance between the two 8-channel
// halves of a K = 16 step, SBO the distance between groups of 8 rows. The halo is stored
// chunk-major, [channel chunk c (4)][y (18)][x (18)][8 channels], so that any 8 consecutive
// pixels of a row - whatever the tap's x shift - form one core matrix: for tap (dy, dx) and
// pixel half h, A is the 128 x 16 block of rows (output row oy, pixels 8h..8h+7) at
// start + ((2 ks) 18 + dy) 18 + dx + 8h (x 16 B), SBO = one halo row (288 B), LBO = one chunk
// (5184 B). B (weights, N = 32 output channels x K) is [tap][c][co][8]: SBO = 128 B, LBO = 512 B.
// Per tile: 2 halves x 9 taps x 2 K steps = 36 MMAs of 128 x 32 x 16 into two 32-column
// accumulators (one 64-column TMEM stage).
constexpr int kHaloChunk = kHalo * kHalo * 8;                 // bf16 elements of one channel chunk
constexpr int kHaloTc = 4 * kHaloChunk;                        // one halo buffer

__device__ __forceinline__ uint64_t umma_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; base offset 0, no swizzle
  return d;
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- Pipelined tcgen05 convolution (warp-specialised). The same BF16 products as k_conv_mid in
// the same FP32 accumulation order per tap (so the same bits), organised as a pipeline without
// block barriers:
//   warp 8 (producer): the halo of each tile into one of kTcHaloStages buffers with cp.async; a
//     stage is handed over (mbarrier `full`) once the lane's copies have landed and been fenced
//     for the tensor cores' (async) proxy, two stages in flight per lane;
//   warp 9, lane 0 (issuer): per tile the 36 tcgen05.mma into one of kTcAccStages TMEM
//     accumulators, then two commits: `accf` (accumulator complete) and `empty` (the halo
//     buffer may be refilled);
//   warps 0..7 (epilogue): tcgen05.ld of the accumulator, `acce` (it may be overwritten), then
//     bias and ReLU (forward) or the ReLU mask (backward data), BF16, global stores.
// Every wait is bounded: one that gives up sets the CTA's failure flag, the other roles leave
// their loops at their next check or bounded wait, the issuer waits (longer, still bounded) for
// its MMAs to complete, and the CTA frees its TMEM and reports the failure.
// Measured on the forward of 8 x 511^2 fields (one CTA per SM): 4 stages handed over one tile
// after their copies were issued 0.624 ms; 4 stages, three tiles after 0.855 ms; 8 stages, five
// tiles after 0.679 ms.
constexpr int kTcHaloStages = 4;
constexpr int kTcLag = 1;          // tiles between issuing a stage's copies and handing it over
constexpr int kTcAccStages = 4;    // 64 TMEM columns each (two halves x 32 channels)
static_assert(kTcLag < kTcHaloStages, "the producer's wait for a free stage needs its MMAs issued");
constexpr int kTcEpiWarps = 8;
constexpr int kTcProducer = 8;
constexpr int kTcIssuer = 9;
constexpr int kTcpThreads = 320;
constexpr int kTcpTmemCols = 64 * kTcAccStages;
constexpr size_t kTcWeightBytes = (size_t)9 * 4 * kC * 8 * sizeof(bf16);
constexpr size_t kTcHaloBytes = (size_t)kHaloTc * sizeof(bf16);
constexpr size_t kTcpSmem = kTcWeightBytes + kTcHaloStages * kTcHaloBytes + 256;  // + barriers, TMEM slot
static_assert(kTcWeightBytes % 128 == 0 && kTcHaloBytes % 16 == 0, "descriptor alignment");
// the last address a tap's descriptor reaches stays inside its halo buffer
static_assert(((size_t)((2 * kHalo + 2) * kHalo + 2 + 8) * 16 + 15 * kHalo * 16 + (size_t)kHaloChunk * 2 + 128) <=
                  kTcHaloBytes,
              "descriptor reach");
// CTAs per SM are limited by shared memory to at most two, so their TMEM (2 x 256 columns) fits
static_assert(3 * (kTcpSmem + 1024) > 228 * 1024 && 2 * kTcpTmemCols <= 512, "TMEM occupancy");
static_assert(kTcpSmem <= 227 * 1024, "shared memory per CTA");

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"((unsigned)__cvta_generic_to_shared(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(
                   (unsigned)__cvta_generic_to_shared(b))
               : "memory");
}
__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__global__ void __launch_bounds__(kTcpThreads, 2) k_conv_mid_tcp(const bf16* __restrict__ x, bf16* __restrict__ y,
                                                                 const bf16* __restrict__ W,
                                                                 const float* __restrict__ bias,
                                                                 const bf16* __restrict__ mask, int S, int tiles_x,
                                                                 int tiles, int mode, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char tcp_smem[];
  bf16* ws = reinterpret_cast<bf16*>(tcp_smem);                       // [tap][c][co][8]
  bf16* halo = reinterpret_cast<bf16*>(tcp_smem + kTcWeightBytes);    // kTcHaloStages buffers
  uint64_t* bars = reinterpret_cast<uint64_t*>(tcp_smem + kTcWeightBytes + kTcHaloStages * kTcHaloBytes);
  uint64_t* full = bars;                        // halo landed: 32 producer arrivals
  uint64_t* empty = bars + kTcHaloStages;       // halo read by the MMAs: one commit
  uint64_t* accf = bars + 2 * kTcHaloStages;    // accumulator complete: one commit
  uint64_t* acce = accf + kTcAccStages;         // accumulator read out: one arrival per epilogue warp
  uint64_t* drain = acce + kTcAccStages;        // every issued MMA complete
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(drain + 1);
  __shared__ volatile int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_img = tiles_x * tiles_x;
  const int count = (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  auto tile_origin = [&](int j, int& img, int& ty0, int& tx0) {
    const int tl = blockIdx.x + j * gridDim.x;
    img = tl / per_img;
    const int r = tl - img * per_img;
    ty0 = (r / tiles_x) * kTile;
    tx0 = (r % tiles_x) * kTile;
  };
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int i = 0; i < kTcHaloStages; ++i) {
      mbar_init(full + i, 32);
      mbar_init(empty + i, 1);
    }
    for (int i = 0; i < kTcAccStages; ++i) {
      mbar_init(accf + i, 1);
      mbar_init(acce + i, kTcEpiWarps);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                 "n"(kTcpTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  for (int c = threadIdx.x; c < 9 * kC * 4; c += kTcpThreads) {
    const int row = c >> 2, part = c & 3;  // row = tap * 32 + output channel, part = channel chunk
    const int tap = row / kC, co = row - tap * kC;
    *reinterpret_cast<uint4*>(ws + ((tap * 4 + part) * kC + co) * 8) =
        *reinterpret_cast<const uint4*>(W + row * kC + part * 8);
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::);  // the weights, for the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const unsigned tmem = *tmem_slot;

  if (warp == kTcProducer) {
    // lane-strided 16-byte copies of the chunk-major halo [chunk][y][x][8] of tile j into stage s
    auto load = [&](int j) {
      int img, ty0, tx0;
      tile_origin(j, img, ty0, tx0);
      bf16* hb = halo + (size_t)(j % kTcHaloStages) * kHaloTc;
      const bf16* xi = x + (size_t)img * S * S * kC;
      for (int c = lane; c < kHalo * kHalo * 4; c += 32) {
        const int pix = c >> 2, part = c & 3;
        const int yy = pix / kHalo, xx = pix - yy * kHalo;
        const int gy = ty0 - 1 + yy, gx = tx0 - 1 + xx;
        const bool in = gy >= 0 && gy < S && gx >= 0 && gx < S;
        const bf16* src = in ? xi + ((size_t)gy * S + gx) * kC + part * 8 : xi;
        cp_async16(hb + part * kHaloChunk + (yy * kHalo + xx) * 8, src, in ? 16 : 0);
      }
      cp_async_commit();
    };
    // A stage is handed over kTcLag tiles after its copies were issued (kTcLag + 1 stages in
    // flight per lane): this lane's copies of it have landed (cp.async groups complete in order)
    // and are fenced for the async proxy.
    auto publish = [&](int j) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::);
      mbar_arrive(full + j % kTcHaloStages);
    };
    int j = 0;
    for (; j < count; ++j) {
      bool ok = true;
      if (j >= kTcHaloStages)
        ok = chwait::mbar_wait(saddr(empty + j % kTcHaloStages), ((j / kTcHaloStages) - 1) & 1, chwait::kSpins);
      if (!__all_sync(0xffffffffu, ok)) s_fail = 1;  // warp-uniform: one lane giving up stops all
      if (s_fail) break;
      load(j);
      if (j >= kTcLag) {
        cp_async_wait<kTcLag>();
        publish(j - kTcLag);
      }
    }
    cp_async_wait<0>();
    if (!s_fail)
      for (int t = (j > kTcLag ? j - kTcLag : 0); t < j; ++t) publish(t);
  } else if (warp == kTcIssuer) {
    if (lane == 0) {
      const unsigned wbase = saddr(ws);
      constexpr uint32_t idesc = umma_idesc(128, 32);
      for (int j = 0; j < count; ++j) {
        const int s = j % kTcHaloStages, a = j % kTcAccStages;
        if (!chwait::mbar_wait(saddr(full + s), (j / kTcHaloStages) & 1, chwait::kSpins)) s_fail = 1;
        if (!s_fail && j >= kTcAccStages &&
            !chwait::mbar_wait(saddr(acce + a), ((j / kTcAccStages) - 1) & 1, chwait::kSpins))
          s_fail = 1;
        if (s_fail) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        const unsigned hbase = saddr(halo + (size_t)s * kHaloTc);
        const unsigned dbase = tmem + 64u * (unsigned)a;
        for (int hh = 0; hh < 2; ++hh)
          for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap - 3 * dy;
            for (int ks = 0; ks < 2; ++ks) {
              const unsigned a_addr = hbase + (unsigned)(((2 * ks * kHalo + dy) * kHalo + dx + 8 * hh) * 16);
              const unsigned b_addr = wbase + (unsigned)((tap * 4 + 2 * ks) * kC * 16);
              const uint64_t ad = umma_desc(a_addr, kHaloChunk * 2, kHalo * 16);
              const uint64_t bd = umma_desc(b_addr, kC * 16, 8 * 16);
              const unsigned acc = (tap | ks) ? 1u : 0u;
              asm volatile(
                  "{\n\t.reg .pred p;\n\t"
                  "setp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dbase + 32u * hh),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            saddr(accf + a)));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            saddr(empty + s)));
      }
      // every MMA issued so far completes before the accumulators are freed
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          saddr(drain)));
      if (!chwait::mbar_wait(saddr(drain), 0u, chwait::kDrainSpins)) s_fail = 1;
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4).. of half h = w / 4 -> pixel (oy, px)
    const int h = warp >> 2, m = (warp & 3) * 32 + lane;
    const int oy = m >> 3, px = 8 * h + (m & 7);
    float bv[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) bv[c] = (mode == 0) ? bias[c] : 0.f;
    for (int j = 0; j < count; ++j) {
      const int a = j % kTcAccStages;
      const bool ok = chwait::mbar_wait(saddr(accf + a), (j / kTcAccStages) & 1, chwait::kSpins);
      if (!__all_sync(0xffffffffu, ok)) s_fail = 1;  // warp-uniform (tcgen05.ld is .sync.aligned)
      if (s_fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      unsigned r[32];
      const unsigned taddr = tmem + ((unsigned)((warp & 3) * 32) << 16) + 64u * (unsigned)a + 32u * h;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
            "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
            "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
      __syncwarp();
      if (lane == 0) mbar_arrive(acce + a);
      int img, ty0, tx0;
      tile_origin(j, img, ty0, tx0);
      const int Y = ty0 + oy, X = tx0 + px;
      if (Y < S && X < S) {
        const size_t o = (size_t)img * S * S * kC + ((size_t)Y * S + X) * kC;
        uint4 mk[4];
        if (mode == 1)
#pragma unroll
          for (int q = 0; q < 4; ++q) mk[q] = *reinterpret_cast<const uint4*>(mask + o + 8 * q);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          unsigned pk[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = 8 * q + 2 * e;
            float v0 = __uint_as_float(r[c]), v1 = __uint_as_float(r[c + 1]);
            if (mode == 0) {
              v0 = fmaxf(v0 + bv[c], 0.f);
              v1 = fmaxf(v1 + bv[c + 1], 0.f);
            } else {
              const __nv_bfloat162 mm = reinterpret_cast<const __nv_bfloat162*>(&mk[q])[e];
              v0 = (__bfloat162float(mm.x) > 0.f) ? v0 : 0.f;
              v1 = (__bfloat162float(mm.y) > 0.f) ? v1 : 0.f;
            }
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v0, v1);
            pk[e] = *reinterpret_cast<const unsigned*>(&b2);
          }
          *reinterpret_cast<uint4*>(y + o + 8 * q) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (s_fail && threadIdx.x == 0) atomicExch(err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kTcpTmemCols));
  }
}

// First layer 1 -> 32: a1 = relu(conv(U, W1) + b1); U FP64 (inference) or FP32 (training).
template <typename TIn>
__global__ void __launch_bounds__(kThreads, 4) k_conv_first(const TIn* __restrict__ u, bf16* __restrict__ y,
                                                         const float* __restrict__ P, int S, float* __restrict__ a0) {
  __shared__ float tile[kHalo * kHalo];
  __shared__ float w[9 * kC + kC];
  const int img = blockIdx.z, ty0 = blockIdx.y * kTile, tx0 = blockIdx.x * kTile;
  const TIn* ui = u + (size_t)img * S * S;
  for (int c = threadIdx.x; c < kHalo * kHalo; c += kThreads) {
    const int yy = c / kHalo, xx = c - yy * kHalo;
    const int gy = ty0 - 1 + yy, gx = tx0 - 1 + xx;
    tile[c] = (gy >= 0 && gy < S && gx >= 0 && gx < S) ? float(ui[(size_t)gy * S + gx]) : 0.f;
  }
  for (int c = threadIdx.x; c < 9 * kC + kC; c += kThreads) w[c] = P[kW1 + c];  // W1 then b1 (contiguous)
  __syncthreads();
  const int oy = threadIdx.x / kTile, ox = threadIdx.x - oy * kTile;
  const int Y = ty0 + oy, X = tx0 + ox;
  if (Y >= S || X >= S) return;
  if (a0) a0[((size_t)img * S + Y) * S + X] = tile[(oy + 1) * kHalo + ox + 1];
  float nb[9];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) nb[tap] = tile[(oy + tap / 3) * kHalo + ox + tap % 3];
  bf16* yo = y + (((size_t)img * S + Y) * S + X) * kC;
  float acc[kC];
#pragma unroll
  for (int co = 0; co < kC; ++co) acc[co] = w[9 * kC + co];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
    for (int co = 0; co < kC; ++co) acc[co] += w[tap * kC + co] * nb[tap];
  }
  // eight channels per 16-byte store (a pixel's 64 bytes in four stores, not sixteen)
#pragma unroll
  for (int c8 = 0; c8 < kC; c8 += 8) {
    unsigned h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float lo = fmaxf(acc[c8 + 2 * q], 0.f), hi = fmaxf(acc[c8 + 2 * q + 1], 0.f);
      h[q] = (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
             ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
    }
    *reinterpret_cast<uint4*>(yo + c8) = make_uint4(h[0], h[1], h[2], h[3]);
  }
}

// Last layer 32 -> 1: r = conv(a5, W6) + b6 (FP32); inference variant writes out = base + r (FP64).
__global__ void __launch_bounds__(kThreads) k_conv_last(const bf16* __restrict__ x, float* __restrict__ r,
                                                        const float* __restrict__ P, int S,
                                                        const double* __restrict__ base, double* __restrict__ out) {
  __shared__ __align__(16) bf16 tile[kHalo * kHalo * kPix];
  __shared__ float w[9 * kC + 1];
  const int img = blockIdx.z, ty0 = blockIdx.y * kTile, tx0 = blockIdx.x * kTile;
  load_halo(tile, x + (size_t)img * S * S * kC, S, ty0, tx0);
  for (int c = threadIdx.x; c < 9 * kC + 1; c += kThreads) w[c] = P[kW6 + c];  // W6 then b6
  __syncthreads();
  const int oy = threadIdx.x / kTile, ox = threadIdx.x - oy * kTile;
  const int Y = ty0 + oy, X = tx0 + ox;
  if (Y >= S || X >= S) return;
  float s = w[9 * kC];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const bf16* p = tile + ((oy + tap / 3) * kHalo + ox + tap % 3) * kPix;
#pragma unroll
    for (int c8 = 0; c8 < kC; c8 += 8) {
      // eight channels per 16-byte shared load (80-byte pixel stride: conflict-free per quarter warp)
      const uint4 raw = *reinterpret_cast<const uint4*>(p + c8);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int ci = c8 + 2 * q;
        const float2 v = __bfloat1622float2(h[q]);
        s += w[tap * kC + ci] * v.x + w[tap * kC + ci + 1] * v.y;
      }
    }
  }
  const size_t o = ((size_t)img * S + Y) * S + X;
  if (r) r[o] = s;
  if (out) out[o] = base[o] + (double)s;
}

// Energy of each crop's target on the window, E_b = sum t^2 + 1e-12 count (one block per crop;
// the floor keeps an all-zero target finite), for the relative loss.
__global__ void k_target_energy(const float* __restrict__ t, int S, int margin, double* __restrict__ eng) {
  __shared__ double sh[kThreads / 32];
  const int inner = S - 2 * margin;
  const float* tb = t + (size_t)blockIdx.x * S * S;
  double acc = 0.0;
  for (int k = threadIdx.x; k < inner * inner; k += kThreads) {
    const float v = tb[(size_t)(margin + k / inner) * S + margin + k % inner];
    acc += (double)v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) s += sh[i];
    eng[blockIdx.x] = s + 1e-12 * inner * inner;
  }
}

// Loss on the window [margin, S - margin)^2, dr = dLoss/dr there and 0 elsewhere; per-block
// partial sums of the loss. eng = null: mean of (r - t)^2 over the batch's windows; otherwise
// the mean over the batch of sum (r - t)^2 / E_b (the relative squared error of each crop).
__global__ void k_loss(const float* __restrict__ r, const float* __restrict__ t, float* __restrict__ dr, int B, int S,
                       int margin, const double* __restrict__ eng, double* __restrict__ part) {
  __shared__ double sh[kThreads / 32];
  const size_t total = (size_t)B * S * S;
  const int inner = S - 2 * margin;
  const double inv = eng ? 1.0 / B : 1.0 / ((double)B * inner * inner);
  double acc = 0.0;
  for (size_t k = blockIdx.x * (size_t)kThreads + threadIdx.x; k < total; k += (size_t)gridDim.x * kThreads) {
    const int X = (int)(k % S), Y = (int)((k / S) % S);
    const bool in = Y >= margin && Y < S - margin && X >= margin && X < S - margin;
    const float d = in ? r[k] - t[k] : 0.f;
    const double w = eng ? 1.0 / eng[k / ((size_t)S * S)] : 1.0;
    dr[k] = (float)(2.0 * d * inv * w);
    acc += (double)d * d * w;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) s += sh[i];
    part[blockIdx.x] = s * inv;
  }
}

__global__ void k_loss_sum(const double* __restrict__ part, int n, float* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = (float)s;
  }
}

// Gradient into the last hidden layer: g5[p][ci] = sum_tap W6[tap][ci] dr[p - (tap - 1)], times
// the ReLU mask of a5.
__global__ void __launch_bounds__(kThreads) k_last_bwd(const float* __restrict__ dr, const bf16* __restrict__ a5,
                                                       bf16* __restrict__ g5, const float* __restrict__ P, int S) {
  __shared__ float tile[kHalo * kHalo];
  __shared__ float w[9 * kC];
  const int img = blockIdx.z, ty0 = blockIdx.y * kTile, tx0 = blockIdx.x * kTile;
  const float* di = dr + (size_t)img * S * S;
  for (int c = threadIdx.x; c < kHalo * kHalo; c += kThreads) {
    const int yy = c / kHalo, xx = c - yy * kHalo;
    const int gy = ty0 - 1 + yy, gx = tx0 - 1 + xx;
    tile[c] = (gy >= 0 && gy < S && gx >= 0 && gx < S) ? di[(size_t)gy * S + gx] : 0.f;
  }
  for (int c = threadIdx.x; c < 9 * kC; c += kThreads) w[c] = P[kW6 + c];
  __syncthreads();
  const int oy = threadIdx.x / kTile, ox = threadIdx.x - oy * kTile;
  const int Y = ty0 + oy, X = tx0 + ox;
  if (Y >= S || X >= S) return;
  // dr at p - (tap - 1) = tile position (oy + 1 - (dy - 1), ox + 1 - (dx - 1)) = (oy + 2 - dy, ox + 2 - dx)
  float nb[9];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) nb[tap] = tile[(oy + 2 - tap / 3) * kHalo + ox + 2 - tap % 3];
  const size_t o = (((size_t)img * S + Y) * S + X) * kC;
#pragma unroll
  for (int ci = 0; ci < kC; ci += 2) {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      s0 += w[tap * kC + ci] * nb[tap];
      s1 += w[tap * kC + ci + 1] * nb[tap];
    }
    const float2 m = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(a5 + o + ci));
    *reinterpret_cast<__nv_bfloat162*>(g5 + o + ci) =
        __floats2bfloat162_rn(m.x > 0.f ? s0 : 0.f, m.y > 0.f ? s1 : 0.f);
  }
}

// Weight gradient of a 32 -> 32 layer over one 16 x 16 tile on the tensor cores:
// partial[tile][tap][co][ci] = sum_p g[p][co] x[p + tap - 1][ci], i.e. per tap the product
// G^T (32 x 256 pixels) X_tap (256 x 32) with K = the tile's pixels in chunks of one output row.
// Warp w owns output block (co 16 (w & 1) .., ci 8 (w >> 1) ..) for all nine taps. Both operands
// are pixel-major in shared memory and are read with ldmatrix.trans. The bias partial
// sum_p g[p][co] follows the 9216 weights.
__device__ __forceinline__ void ldsm_x4_t(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned& r0, unsigned& r1, const void* p) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

__global__ void __launch_bounds__(kThreads) k_wgrad_mid(const bf16* __restrict__ g, const bf16* __restrict__ x,
                                                        float* __restrict__ part, int S) {
  __shared__ __align__(16) bf16 tile[kHalo * kHalo * kPix];
  __shared__ __align__(16) bf16 gt[kTile * kTile * kPix];
  const int img = blockIdx.z, ty0 = blockIdx.y * kTile, tx0 = blockIdx.x * kTile;
  const size_t off = (size_t)img * S * S * kC;
  load_halo(tile, x + off, S, ty0, tx0);
  for (int c = threadIdx.x; c < kTile * kTile * 4; c += kThreads) {
    const int pix = c >> 2, part4 = c & 3;
    const int Y = ty0 + pix / kTile, X = tx0 + pix % kTile;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (Y < S && X < S) v = *reinterpret_cast<const uint4*>(g + off + ((size_t)Y * S + X) * kC + part4 * 8);
    *reinterpret_cast<uint4*>(gt + pix * kPix + part4 * 8) = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int co0 = (warp & 1) * 16, ci0 = (warp >> 1) * 8;
  const int mat = lane >> 3, i8 = lane & 7;
  float acc[9][4];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[tap][q] = 0.f;
  for (int oy = 0; oy < kTile; ++oy) {  // K chunk: the 16 pixels of output row oy
    unsigned a[4];
    // A = G^T block (co0.. co0+15, pixels): matrix m reads pixels (m >> 1) * 8 + i8, columns
    // co0 + (m & 1) * 8
    ldsm_x4_t(a[0], a[1], a[2], a[3], gt + (oy * kTile + (mat >> 1) * 8 + i8) * kPix + co0 + (mat & 1) * 8);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3, dx = tap - 3 * dy;
      // B = X_tap block (pixels, ci0.. ci0+7): lanes 0-7 rows of pixels 0-7, lanes 8-15 pixels 8-15
      const int px = ((mat & 1) * 8 + i8);
      unsigned b0, b1;
      ldsm_x2_t(b0, b1, tile + ((oy + dy) * kHalo + px + dx) * kPix + ci0);
      mma16816(acc[tap], a, b0, b1);
    }
  }
  const size_t tileid = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  float* pp = part + tileid * (9 * kC * kC + kC);
  const int gq = lane >> 2, t = lane & 3;
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    float* o = pp + (size_t)tap * kC * kC;
    o[(co0 + gq) * kC + ci0 + 2 * t] = acc[tap][0];
    o[(co0 + gq) * kC + ci0 + 2 * t + 1] = acc[tap][1];
    o[(co0 + gq + 8) * kC + ci0 + 2 * t] = acc[tap][2];
    o[(co0 + gq + 8) * kC + ci0 + 2 * t + 1] = acc[tap][3];
  }
  // bias: 8 threads per output channel, pixels strided by 8, then a shuffle tree
  const int co = threadIdx.x >> 3, sub = threadIdx.x & 7;
  float bsum = 0.f;
  for (int pix = sub; pix < kTile * kTile; pix += 8) bsum += __bfloat162float(gt[pix * kPix + co]);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
  if (sub == 0) pp[9 * kC * kC + co] = bsum;
}

// Weight gradients of the first layer (x = a0 scalar, g = gz1 [32]) or the last (x = a5 [32],
// g = dr scalar) over one tile: 288 weights + bias per tile.
__global__ void __launch_bounds__(kThreads) k_wgrad_edge(const float* __restrict__ a0, const bf16* __restrict__ g1,
                                                         const float* __restrict__ dr, const bf16* __restrict__ a5,
                                                         float* __restrict__ part, int S, int first) {
  __shared__ __align__(16) bf16 tile[kHalo * kHalo * kPix];
  __shared__ float ft[kHalo * kHalo];
  __shared__ __align__(16) bf16 gt[kTile * kTile * kPix];
  __shared__ float fg[kTile * kTile];
  const int img = blockIdx.z, ty0 = blockIdx.y * kTile, tx0 = blockIdx.x * kTile;
  const size_t s2 = (size_t)S * S;
  if (first) {
    for (int c = threadIdx.x; c < kHalo * kHalo; c += kThreads) {
      const int yy = c / kHalo, xx = c - yy * kHalo;
      const int gy = ty0 - 1 + yy, gx = tx0 - 1 + xx;
      ft[c] = (gy >= 0 && gy < S && gx >= 0 && gx < S) ? a0[img * s2 + (size_t)gy * S + gx] : 0.f;
    }
    for (int c = threadIdx.x; c < kTile * kTile * 4; c += kThreads) {
      const int pix = c >> 2, part4 = c & 3;
      const int Y = ty0 + pix / kTile, X = tx0 + pix % kTile;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (Y < S && X < S) v = *reinterpret_cast<const uint4*>(g1 + (img * s2 + (size_t)Y * S + X) * kC + part4 * 8);
      *reinterpret_cast<uint4*>(gt + pix * kPix + part4 * 8) = v;
    }
  } else {
    load_halo(tile, a5 + img * s2 * kC, S, ty0, tx0);
    for (int c = threadIdx.x; c < kTile * kTile; c += kThreads) {
      const int Y = ty0 + c / kTile, X = tx0 + c % kTile;
      fg[c] = (Y < S && X < S) ? dr[img * s2 + (size_t)Y * S + X] : 0.f;
    }
  }
  __syncthreads();
  const size_t tileid = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  float* pp = part + tileid * (9 * kC + kC);
  for (int o = threadIdx.x; o < 9 * kC + kC; o += kThreads) {
    float acc = 0.f;
    if (o < 9 * kC) {
      const int tap = o / kC, c = o - tap * kC;  // first: c = output channel; last: c = input channel
      for (int pix = 0; pix < kTile * kTile; ++pix) {
        const int oy = pix / kTile, ox = pix - oy * kTile;
        const int hp = (oy + tap / 3) * kHalo + ox + tap % 3;
        if (first) acc += __bfloat162float(gt[pix * kPix + c]) * ft[hp];
        else acc += fg[pix] * __bfloat162float(tile[hp * kPix + c]);
      }
    } else {
      const int c = o - 9 * kC;
      for (int pix = 0; pix < kTile * kTile; ++pix)
        acc += first ? __bfloat162float(gt[pix * kPix + c]) : (c == 0 ? fg[pix] : 0.f);
    }
    pp[o] = acc;
  }
}

// Sum over tiles of part[tile * stride + j], j < len, in two fixed-order levels: chunks of
// kChunk tiles (blockIdx.y) into part2[chunk][len], then the chunks (k_reduce); the weights
// (j < wlen) go to grad[dst_w + j], the biases to grad[dst_b + j - wlen].
constexpr int kChunk = 32;
__global__ void k_reduce_chunks(const float* __restrict__ part, int tiles, int stride, int len,
                                double* __restrict__ part2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= len) return;
  const int t0 = blockIdx.y * kChunk, t1 = min(tiles, t0 + kChunk);
  double s = 0.0;
  for (int tl = t0; tl < t1; ++tl) s += part[(size_t)tl * stride + j];
  part2[(size_t)blockIdx.y * len + j] = s;
}

__global__ void k_reduce(const double* __restrict__ part2, int chunks, int len, float* __restrict__ grad, int dst_w,
                         int wlen, int dst_b) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= len) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += part2[(size_t)c * len + j];
  if (j < wlen) grad[dst_w + j] = (float)s;
  else grad[dst_b + (j - wlen)] = (float)s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// BF16 weights of the 32 -> 32 layers: forward [tap][co][ci]; backward data [tap'][ci][co] with
// tap' = 8 - tap (flipped taps, swapped channels).
__global__ void k_pack(const float* __restrict__ P, bf16* __restrict__ wf, bf16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * 9 * kC * kC) return;
  const int l = i / (9 * kC * kC), r = i - l * 9 * kC * kC;
  const int tap = r / (kC * kC), co = (r / kC) % kC, ci = r % kC;
  const float w = P[kW2 + l * kMidStride + r];
  wf[i] = __float2bfloat16_rn(w);
  wb[(size_t)l * 9 * kC * kC + ((8 - tap) * kC + ci) * kC + co] = __float2bfloat16_rn(w);
}

// Random crops of pairs: in = states[t][s] on [y0, y0+S) x [x0, x0+S) (0 outside the grid),
// target = states[t][s + stride] - base[t][s] there (base = states when null).
__global__ void k_crops(const double* __restrict__ states, const double* __restrict__ base,
                        const int4* __restrict__ crops, int nsnap, int n, int stride, int S, float* __restrict__ in,
                        float* __restrict__ tgt) {
  const int b = blockIdx.y;
  const int4 c = crops[b];  // (traj, snap, y0, x0)
  const size_t off = ((size_t)c.x * nsnap + c.y) * n * n;
  const size_t off2 = ((size_t)c.x * nsnap + c.y + stride) * n * n;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S * S; k += gridDim.x * blockDim.x) {
    const int yy = k / S, xx = k - yy * S;
    const int Y = c.z + yy, X = c.w + xx;
    double a = 0.0, t = 0.0;
    if (Y >= 0 && Y < n && X >= 0 && X < n) {
      a = states[off + (size_t)Y * n + X];
      t = states[off2 + (size_t)Y * n + X] - (base ? base[off + (size_t)Y * n + X] : a);
    }
    in[(size_t)b * S * S + k] = (float)a;
    tgt[(size_t)b * S * S + k] = (float)t;
  }
}

// tcgen05 launch of the 32 -> 32 convolution (persistent, like k_conv_mid).
void conv_mid_tc(const bf16* x, bf16* y, const bf16* W, const float* bias, const bf16* mask, int batch, int S,
                 int mode, int* err, cudaStream_t st) {
  static std::mutex mu;
  static std::map<unsigned long long, int> slot_of;  // resident CTAs per context
  int dev = 0;
  cudaGetDevice(&dev);
  std::unique_lock<std::mutex> lock(mu);
  int& slots = slot_of[chctx::cache_key()];
  if (slots == 0) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // One CTA per SM (measured: two per SM take 128 us per layer against 106 us for one); its
    // shared memory admits at most two, so their TMEM (2 x 256 columns) would always fit.
    cudaFuncSetAttribute(k_conv_mid_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcpSmem);
    slots = std::max(1, sms);
  }
  const int tx = (S + kTile - 1) / kTile, tiles = tx * tx * batch;
  const int grid = std::min(tiles, slots);
  lock.unlock();
  k_conv_mid_tcp<<<grid, kTcpThreads, kTcpSmem, st>>>(x, y, W, bias, mask, S, tx, tiles, mode, err);
}

// Persistent launch of k_conv_mid: as many CTAs as fit on the GPU (at most one per tile).
void conv_mid(const bf16* x, bf16* y, const bf16* W, const float* bias, const bf16* mask, int batch, int S, int mode,
              cudaStream_t st) {
  static std::mutex mu;
  static std::map<unsigned long long, int> slot_of;  // resident CTAs of k_conv_mid per context
  int dev = 0;
  cudaGetDevice(&dev);
  std::unique_lock<std::mutex> lock(mu);
  int& slots = slot_of[chctx::cache_key()];
  if (slots == 0) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_conv_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConvSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_mid, kThreads, kConvSmem);
    slots = std::max(1, sms * std::max(1, per_sm));
  }
  const int tx = (S + kTile - 1) / kTile, tiles = tx * tx * batch;
  const int grid = std::min(tiles, slots);
  lock.unlock();
  k_conv_mid<<<grid, kThreads, kConvSmem, st>>>(x, y, W, bias, mask, S, tx, tiles, mode);
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

// --------------------------------------------------------------------------- GTheta

cudaError_t GTheta::init(unsigned long long seed, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b);
  };
  al((void**)&master_, kParams * sizeof(float));
  al((void**)&grad_, kParams * sizeof(float));
  al((void**)&m_, kParams * sizeof(float));
  al((void**)&v_, kParams * sizeof(float));
  al((void**)&wmid_, 4 * 9 * kC * kC * sizeof(bf16));
  al((void**)&wbwd_, 4 * 9 * kC * kC * sizeof(bf16));
  al((void**)&lpart_, 1024 * sizeof(double));
  al((void**)&err_, sizeof(int));
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(err_, 0, sizeof(int), st)) != cudaSuccess) return e;
  // The 32 -> 32 layers run on tcgen05.mma (k_conv_mid_tcp); CH_GTHETA_CONV=mma selects the
  // warp-level mma.sync kernel (k_conv_mid), which gives the same bits
  const char* cv = std::getenv("CH_GTHETA_CONV");
  tc_ = !(cv && std::strcmp(cv, "mma") == 0);
  // He-normal initial weights (Box-Muller on SplitMix64), zero biases; the last layer scaled 0.1
  std::vector<float> p(kParams, 0.f);
  const int cin[6] = {1, 32, 32, 32, 32, 32}, cout[6] = {32, 32, 32, 32, 32, 1};
  uint64_t s = seed;
  for (int l = 0; l < 6; ++l) {
    const double sd = std::sqrt(2.0 / (9.0 * cin[l])) * (l == 5 ? 0.1 : 1.0);
    for (int i = 0; i < 9 * cout[l] * cin[l]; ++i) {
      const double u1 = ((splitmix(s) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
      const double u2 = (splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
      p[kOffW[l] + i] = float(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2));
    }
  }
  return set_params(p.data(), st);
}

void GTheta::release() {
  void* ptrs[] = {master_, grad_, m_, v_, wmid_, wbwd_, loss_dev_, a0_, r_, dr_, part_, tgt_, crops_, lpart_,
                  act_[0], act_[1], act_[2], act_[3], act_[4], g_[0], g_[1], part2_, err_, eng_};
  for (void* q : ptrs) cudaFree(q);
  master_ = grad_ = m_ = v_ = nullptr;
  wmid_ = wbwd_ = nullptr;
  loss_dev_ = a0_ = r_ = dr_ = part_ = tgt_ = nullptr;
  part2_ = nullptr;
  err_ = nullptr;
  crops_ = nullptr;
  lpart_ = nullptr;
  eng_ = nullptr;
  for (auto& a : act_) a = nullptr;
  for (auto& gg : g_) gg = nullptr;
  cap_batch_ = cap_S_ = 0;
}

cudaError_t GTheta::refresh_bf16(cudaStream_t st) {
  k_pack<<<(4 * 9 * kC * kC + 255) / 256, 256, 0, st>>>(master_, wmid_, wbwd_);
  return cudaGetLastError();
}

cudaError_t GTheta::set_params(const float* host, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(master_, host, kParams * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m_, 0, kParams * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(v_, 0, kParams * sizeof(float), st);
  adam_t_ = 0;
  if (e == cudaSuccess) e = refresh_bf16(st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t GTheta::get_params(float* host, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(host, master_, kParams * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t GTheta::ensure(int batch, int S) {
  if (batch <= cap_batch_ && S <= cap_S_) return cudaSuccess;
  const int B = std::max(batch, cap_batch_), SS = std::max(S, cap_S_);
  void* old[] = {a0_, r_, dr_, tgt_, act_[0], act_[1], act_[2], act_[3], act_[4], g_[0], g_[1], part_, crops_, part2_,
                 eng_};
  for (void* q : old) cudaFree(q);
  const size_t f = (size_t)B * SS * SS;
  const size_t tiles = (size_t)B * ((SS + kTile - 1) / kTile) * ((SS + kTile - 1) / kTile);
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b);
  };
  al((void**)&a0_, f * sizeof(float));
  al((void**)&r_, f * sizeof(float));
  al((void**)&dr_, f * sizeof(float));
  al((void**)&tgt_, f * sizeof(float));
  for (auto& a : act_) al((void**)&a, f * kC * sizeof(bf16));
  for (auto& gg : g_) al((void**)&gg, f * kC * sizeof(bf16));
  part_cap_ = tiles * (9 * kC * kC + kC);
  al((void**)&part_, part_cap_ * sizeof(float));
  al((void**)&part2_, ((tiles + kChunk - 1) / kChunk) * (size_t)(9 * kC * kC + kC) * sizeof(double));
  al((void**)&crops_, (size_t)B * sizeof(int4));
  al((void**)&eng_, (size_t)B * sizeof(double));
  if (e == cudaSuccess) {
    cap_batch_ = B;
    cap_S_ = SS;
  }
  return e;
}

cudaError_t GTheta::ensure_losses(int count, cudaStream_t st) {
  if (count <= loss_cap_) return cudaSuccess;
  const int cap = std::max(count, 2 * loss_cap_);
  float* p = nullptr;
  cudaError_t e = cudaMalloc(&p, cap * sizeof(float));
  if (e == cudaSuccess && loss_cap_ > 0)
    e = cudaMemcpyAsync(p, loss_dev_, loss_cap_ * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(p);
    return e;
  }
  cudaFree(loss_dev_);
  loss_dev_ = p;
  loss_cap_ = cap;
  return cudaSuccess;
}

cudaError_t GTheta::forward_acts(const void* in, bool in64, int batch, int S, cudaStream_t st) {
  const dim3 grid((S + kTile - 1) / kTile, (S + kTile - 1) / kTile, batch);
  if (in64) k_conv_first<double><<<grid, kThreads, 0, st>>>((const double*)in, act_[0], master_, S, nullptr);
  else  // keep a copy of the input for the first layer's weight gradient (unless it already is a0_)
    k_conv_first<float><<<grid, kThreads, 0, st>>>((const float*)in, act_[0], master_, S,
                                                   in == a0_ ? nullptr : a0_);
  for (int l = 0; l < 4; ++l)
    if (tc_)
      conv_mid_tc(act_[l], act_[l + 1], wmid_ + (size_t)l * 9 * kC * kC, master_ + kOffB[l + 1], nullptr, batch, S,
                  0, err_, st);
    else
      conv_mid(act_[l], act_[l + 1], wmid_ + (size_t)l * 9 * kC * kC, master_ + kOffB[l + 1], nullptr, batch, S, 0,
               st);
  return cudaGetLastError();
}

__global__ void k_bf16_to_f32(const bf16* __restrict__ in, float* __restrict__ out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = __bfloat162float(in[i]);
}

cudaError_t GTheta::activations(const double* in, int batch, int S, float* out, cudaStream_t st) {
  cudaError_t e = ensure(batch, S);
  if (e != cudaSuccess) return e;
  e = forward_acts(in, true, batch, S, st);
  if (e != cudaSuccess) return e;
  const size_t per = (size_t)batch * S * S * kC;
  for (int l = 0; l < 5; ++l) k_bf16_to_f32<<<1024, 256, 0, st>>>(act_[l], out + l * per, per);
  const dim3 grid((S + kTile - 1) / kTile, (S + kTile - 1) / kTile, batch);
  k_conv_last<<<grid, kThreads, 0, st>>>(act_[4], out + 5 * per, master_, S, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t GTheta::forward64(const double* in, const double* base, double* out, int batch, int S,
                              cudaStream_t st) {
  cudaError_t e = ensure(batch, S);
  if (e != cudaSuccess) return e;
  e = forward_acts(in, true, batch, S, st);
  if (e != cudaSuccess) return e;
  const dim3 grid((S + kTile - 1) / kTile, (S + kTile - 1) / kTile, batch);
  k_conv_last<<<grid, kThreads, 0, st>>>(act_[4], nullptr, master_, S, base ? base : in, out);
  return cudaGetLastError();
}

void GTheta::reduce_tiles(int tiles, int stride, int len, int dst_w, int wlen, int dst_b, cudaStream_t st) {
  const int chunks = (tiles + kChunk - 1) / kChunk;
  k_reduce_chunks<<<dim3((len + 255) / 256, chunks), 256, 0, st>>>(part_, tiles, stride, len, part2_);
  k_reduce<<<(len + 255) / 256, 256, 0, st>>>(part2_, chunks, len, grad_, dst_w, wlen, dst_b);
}

cudaError_t GTheta::grad_step(const float* in, const float* target, int batch, int S, int margin, int slot,
                              cudaStream_t st) {
  cudaError_t e = ensure(batch, S);
  if (e != cudaSuccess) return e;
  if ((e = ensure_losses(slot + 1, st)) != cudaSuccess) return e;
  const dim3 grid((S + kTile - 1) / kTile, (S + kTile - 1) / kTile, batch);
  const int tiles = grid.x * grid.y * grid.z;
  e = forward_acts(in, false, batch, S, st);
  if (e != cudaSuccess) return e;
  k_conv_last<<<grid, kThreads, 0, st>>>(act_[4], r_, master_, S, nullptr, nullptr);
  const int lb = 256;
  if (rel_loss_) k_target_energy<<<batch, kThreads, 0, st>>>(target, S, margin, eng_);
  k_loss<<<lb, kThreads, 0, st>>>(r_, target, dr_, batch, S, margin, rel_loss_ ? eng_ : nullptr, lpart_);
  k_loss_sum<<<1, 32, 0, st>>>(lpart_, lb, loss_dev_ + slot);
  // last layer: weights from (dr, a5), gradient into a5
  const int le = 9 * kC + kC;
  k_wgrad_edge<<<grid, kThreads, 0, st>>>(nullptr, nullptr, dr_, act_[4], part_, S, 0);
  reduce_tiles(tiles, le, 9 * kC + 1, kOffW[5], 9 * kC, kOffB[5], st);
  k_last_bwd<<<grid, kThreads, 0, st>>>(dr_, act_[4], g_[0], master_, S);
  // 32 -> 32 layers 5, 4, 3, 2 (indices l + 1 = 4..1): weights from (g, input activation), then
  // gradient through the layer into the activation below (masked by its ReLU)
  int cur = 0;
  const int lm = 9 * kC * kC + kC;
  for (int l = 3; l >= 0; --l) {
    k_wgrad_mid<<<grid, kThreads, 0, st>>>(g_[cur], act_[l], part_, S);
    reduce_tiles(tiles, lm, lm, kOffW[l + 1], 9 * kC * kC, kOffB[l + 1], st);
    if (tc_)
      conv_mid_tc(g_[cur], g_[cur ^ 1], wbwd_ + (size_t)l * 9 * kC * kC, nullptr, act_[l], batch, S, 1, err_, st);
    else
      conv_mid(g_[cur], g_[cur ^ 1], wbwd_ + (size_t)l * 9 * kC * kC, nullptr, act_[l], batch, S, 1, st);
    cur ^= 1;
  }
  // first layer: weights from (g1, a0)
  k_wgrad_edge<<<grid, kThreads, 0, st>>>(a0_, g_[cur], nullptr, nullptr, part_, S, 1);
  reduce_tiles(tiles, le, le, kOffW[0], 9 * kC, kOffB[0], st);
  return cudaGetLastError();
}

cudaError_t GTheta::train(const double* states, const double* base, int ntraj, int nsnap, int n, int stride,
                          int steps, int batch, double lr, unsigned long long seed, cudaStream_t st) {
  // Crops of 76 x 76 with the loss on the central 64 x 64: the 13 x 13 receptive field of the
  // window stays inside the crop. A grid smaller than the window is taken whole (S = n + 12).
  const int margin = kTrainMargin, S = train_crop(n);
  if (nsnap <= stride || ntraj < 1 || steps < 1 || batch < 1) return cudaErrorInvalidValue;
  cudaError_t e = ensure(batch, S);
  if (e == cudaSuccess) e = ensure_losses(steps, st);
  if (e != cudaSuccess) return e;
  std::vector<int4> crops(batch);
  uint64_t s = seed;
  const int span = n + 2 * margin - S + 1;  // crop origins in [-margin, n + margin - S]
  for (int it = 0; it < steps && e == cudaSuccess; ++it) {
    chtrace::Range range("training step");
    for (int b = 0; b < batch; ++b) {
      crops[b].x = (int)(splitmix(s) % (uint64_t)ntraj);
      crops[b].y = (int)(splitmix(s) % (uint64_t)(nsnap - stride));
      crops[b].z = (int)(splitmix(s) % (uint64_t)std::max(span, 1)) - margin;
      crops[b].w = (int)(splitmix(s) % (uint64_t)std::max(span, 1)) - margin;
    }
    e = cudaMemcpyAsync(crops_, crops.data(), batch * sizeof(int4), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) break;
    k_crops<<<dim3((S * S + 255) / 256, batch), 256, 0, st>>>(states, base, crops_, nsnap, n, stride, S, a0_,
                                                                       tgt_);
    // a0_ doubles as the crop input buffer: k_conv_first re-writes the same values into it
    e = grad_step(a0_, tgt_, batch, S, margin, it, st);
    if (e != cudaSuccess) break;
    ++adam_t_;
    const float c1 = 1.f - std::pow(0.9f, (float)adam_t_), c2 = 1.f - std::pow(0.999f, (float)adam_t_);
    k_adam<<<(kParams + 255) / 256, 256, 0, st>>>(master_, grad_, m_, v_, kParams, (float)lr, c1, c2);
    e = refresh_bf16(st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

int GTheta::wait_failures(cudaStream_t st) {
  int v = 0;
  if (cudaMemcpyAsync(&v, err_, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return 1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return 1;
  return v;
}

cudaError_t GTheta::read_losses(float* host, int count, cudaStream_t st) {
  if (count > loss_cap_) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyAsync(host, loss_dev_, count * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

}  // namespace chg3
