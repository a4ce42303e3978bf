// Batched pentadiagonal solver for one system per CTA (sm_103a).
//
// The implicit steps of Section 2.1 (Eq. 2.3-2.5) need, per time step, a solve with
//   I + eps^2 dt D_h^2 + c dt (-D_h) diag(w)
// which in 1D is pentadiagonal (D_h of Eq. 3.2 is tridiagonal). Pairing rows (2i, 2i+1)
// turns it into a block-tridiagonal system with 2x2 blocks A_i x_{i-1} + B_i x_i + C_i x_{i+1}
// = d_i. A CTA of T threads owns one system; thread t holds P consecutive block rows in
// registers. The solve is a partition method:
//   1. each thread eliminates the interior block rows of its chunk (block Thomas), writing
//      its first and last interior unknowns as affine functions of the two separator
//      unknowns (the first block row of its own chunk and of the next chunk);
//   2. the T separator unknowns satisfy a block-tridiagonal system, solved by block parallel
//      cyclic reduction across the CTA (log2 T levels in shared memory);
//   3. each thread back-substitutes its interior rows.
// Work is O(n) (about 90 flops per row), independent of the number of threads except for the
// T-row reduced system. No pivoting: the matrices are I plus a positive-definite fourth
// difference plus a small convective part, and the partition method then behaves as
// Gaussian elimination without pivoting on a positive-definite-dominated matrix.
#pragma once
#include <cuda_runtime.h>

namespace chg {

template <typename S>
struct M2 {
  S a, b, c, d;  // [[a b], [c d]]
};
template <typename S>
struct V2 {
  S x, y;
};

template <typename S>
__device__ __forceinline__ M2<S> mmul(const M2<S>& p, const M2<S>& q) {
  return {p.a * q.a + p.b * q.c, p.a * q.b + p.b * q.d, p.c * q.a + p.d * q.c, p.c * q.b + p.d * q.d};
}
template <typename S>
__device__ __forceinline__ V2<S> mvec(const M2<S>& p, const V2<S>& v) {
  return {p.a * v.x + p.b * v.y, p.c * v.x + p.d * v.y};
}
template <typename S>
__device__ __forceinline__ M2<S> madd(const M2<S>& p, const M2<S>& q) {
  return {p.a + q.a, p.b + q.b, p.c + q.c, p.d + q.d};
}
template <typename S>
__device__ __forceinline__ M2<S> msub(const M2<S>& p, const M2<S>& q) {
  return {p.a - q.a, p.b - q.b, p.c - q.c, p.d - q.d};
}
template <typename S>
__device__ __forceinline__ M2<S> mneg(const M2<S>& p) {
  return {-p.a, -p.b, -p.c, -p.d};
}
template <typename S>
__device__ __forceinline__ V2<S> vadd(const V2<S>& p, const V2<S>& q) {
  return {p.x + q.x, p.y + q.y};
}
template <typename S>
__device__ __forceinline__ V2<S> vsub(const V2<S>& p, const V2<S>& q) {
  return {p.x - q.x, p.y - q.y};
}
template <typename S>
__device__ __forceinline__ M2<S> minv(const M2<S>& p) {
  const S r = S(1) / (p.a * p.d - p.b * p.c);
  return {p.d * r, -p.b * r, -p.c * r, p.a * r};
}
template <typename S>
__device__ __forceinline__ M2<S> mzero() {
  return {S(0), S(0), S(0), S(0)};
}

// Shared memory of the solver: reduced system in structure-of-arrays form.
template <typename S, int T>
struct SolverSmem {
  S red[14][T];  // RA(4) RB(4) RC(4) Rd(2) of the reduced (separator) system
  S nbr[10][T];  // last-interior representation of each chunk: g(2) G(4) H(4)
  S sep[2][T];   // separator unknowns
};

template <typename S, int T>
__device__ __forceinline__ void put_m(S (*arr)[T], int base, int t, const M2<S>& m) {
  arr[base + 0][t] = m.a;
  arr[base + 1][t] = m.b;
  arr[base + 2][t] = m.c;
  arr[base + 3][t] = m.d;
}
template <typename S, int T>
__device__ __forceinline__ M2<S> get_m(S (*arr)[T], int base, int t) {
  return {arr[base + 0][t], arr[base + 1][t], arr[base + 2][t], arr[base + 3][t]};
}

// Warp shuffles of the 2x2 blocks and 2-vectors: a CTA of one warp exchanges through these
// instead of shared memory and block barriers (out-of-range lanes get their own values back,
// which the callers do not use).
template <typename S>
__device__ __forceinline__ V2<S> shfl_up_v(const V2<S>& v, int s) {
  return {__shfl_up_sync(0xffffffffu, v.x, s), __shfl_up_sync(0xffffffffu, v.y, s)};
}
template <typename S>
__device__ __forceinline__ V2<S> shfl_down_v(const V2<S>& v, int s) {
  return {__shfl_down_sync(0xffffffffu, v.x, s), __shfl_down_sync(0xffffffffu, v.y, s)};
}
template <typename S>
__device__ __forceinline__ M2<S> shfl_up_m(const M2<S>& m, int s) {
  return {__shfl_up_sync(0xffffffffu, m.a, s), __shfl_up_sync(0xffffffffu, m.b, s),
          __shfl_up_sync(0xffffffffu, m.c, s), __shfl_up_sync(0xffffffffu, m.d, s)};
}
template <typename S>
__device__ __forceinline__ M2<S> shfl_down_m(const M2<S>& m, int s) {
  return {__shfl_down_sync(0xffffffffu, m.a, s), __shfl_down_sync(0xffffffffu, m.b, s),
          __shfl_down_sync(0xffffffffu, m.c, s), __shfl_down_sync(0xffffffffu, m.d, s)};
}

// Solve the block-tridiagonal system held as (A[l], B[l], C[l], d[l]), l = 0..P-1 of thread t
// (block row t*P + l). Block rows beyond the system are identity rows with zero couplings.
// On return x[l] holds the solution. All threads of the CTA must call this.
template <typename S, int T, int P>
__device__ void block_tridiag_solve(const M2<S> (&A)[P], const M2<S> (&B)[P], const M2<S> (&C)[P],
                                    const V2<S> (&d)[P], V2<S> (&x)[P], SolverSmem<S, T>& sm) {
  const int t = threadIdx.x;
  // ---- 1. local elimination of interior block rows l = 1..P-1
  M2<S> Binv[P];
  M2<S> Et[P];
  V2<S> dd[P];
  M2<S> RA, RB, RC;
  V2<S> Rd;
  if constexpr (P >= 2) {
    M2<S> Bt = B[1];
    Et[1] = A[1];
    dd[1] = d[1];
#pragma unroll
    for (int l = 2; l < P; ++l) {
      Binv[l - 1] = minv(Bt);
      const M2<S> L = mmul(A[l], Binv[l - 1]);
      Bt = msub(B[l], mmul(L, C[l - 1]));
      dd[l] = vsub(d[l], mvec(L, dd[l - 1]));
      Et[l] = mneg(mmul(L, Et[l - 1]));
    }
    Binv[P - 1] = minv(Bt);
    // backward recurrence: x_l = g + G S_t + H S_{t+1}
    V2<S> g = mvec(Binv[P - 1], dd[P - 1]);
    M2<S> G = mneg(mmul(Binv[P - 1], Et[P - 1]));
    M2<S> H = mneg(mmul(Binv[P - 1], C[P - 1]));
    // publish the last-interior representation for thread t+1 (one warp: shuffles)
    V2<S> gL;
    M2<S> GL, HL;
    if constexpr (T == 32) {
      gL = shfl_up_v(g, 1);
      GL = shfl_up_m(G, 1);
      HL = shfl_up_m(H, 1);
    } else {
      sm.nbr[0][t] = g.x;
      sm.nbr[1][t] = g.y;
      put_m<S, T>(sm.nbr, 2, t, G);
      put_m<S, T>(sm.nbr, 6, t, H);
    }
#pragma unroll
    for (int l = P - 2; l >= 1; --l) {
      g = mvec(Binv[l], vsub(dd[l], mvec(C[l], g)));
      G = mneg(mmul(Binv[l], madd(Et[l], mmul(C[l], G))));
      H = mneg(mmul(Binv[l], mmul(C[l], H)));
    }
    if constexpr (T != 32) __syncthreads();
    // reduced row of separator t: A0 x_{i0-1} + B0 S_t + C0 x_{i0+1} = d0
    RB = madd(B[0], mmul(C[0], G));
    Rd = vsub(d[0], mvec(C[0], g));
    RC = mmul(C[0], H);
    RA = mzero<S>();
    if (t > 0) {
      if constexpr (T != 32) {
        gL = {sm.nbr[0][t - 1], sm.nbr[1][t - 1]};
        GL = get_m<S, T>(sm.nbr, 2, t - 1);
        HL = get_m<S, T>(sm.nbr, 6, t - 1);
      }
      RA = mmul(A[0], GL);
      RB = madd(RB, mmul(A[0], HL));
      Rd = vsub(Rd, mvec(A[0], gL));
    }
  } else {
    RA = A[0];
    RB = B[0];
    RC = C[0];
    Rd = d[0];
  }
  // ---- 2. block parallel cyclic reduction on the T separators
#pragma unroll 1
  for (int s = 1; s < T; s <<= 1) {
    M2<S> nA = mzero<S>(), nC = mzero<S>();
    M2<S> nB = RB;
    V2<S> nd = Rd;
    if constexpr (T == 32) {
      // the rows of separators t - s and t + s by shuffles (one warp)
      const M2<S> Am = shfl_up_m(RA, s), Bm = shfl_up_m(RB, s), Cm = shfl_up_m(RC, s);
      const V2<S> dm = shfl_up_v(Rd, s);
      const M2<S> Ap = shfl_down_m(RA, s), Bp = shfl_down_m(RB, s), Cp = shfl_down_m(RC, s);
      const V2<S> dp = shfl_down_v(Rd, s);
      if (t - s >= 0) {
        const M2<S> al = mneg(mmul(RA, minv(Bm)));
        nA = mmul(al, Am);
        nB = madd(nB, mmul(al, Cm));
        nd = vadd(nd, mvec(al, dm));
      }
      if (t + s < T) {
        const M2<S> ga = mneg(mmul(RC, minv(Bp)));
        nC = mmul(ga, Cp);
        nB = madd(nB, mmul(ga, Ap));
        nd = vadd(nd, mvec(ga, dp));
      }
    } else {
      put_m<S, T>(sm.red, 0, t, RA);
      put_m<S, T>(sm.red, 4, t, RB);
      put_m<S, T>(sm.red, 8, t, RC);
      sm.red[12][t] = Rd.x;
      sm.red[13][t] = Rd.y;
      __syncthreads();
      if (t - s >= 0) {
        const M2<S> al = mneg(mmul(RA, minv(get_m<S, T>(sm.red, 4, t - s))));
        nA = mmul(al, get_m<S, T>(sm.red, 0, t - s));
        nB = madd(nB, mmul(al, get_m<S, T>(sm.red, 8, t - s)));
        nd = vadd(nd, mvec(al, V2<S>{sm.red[12][t - s], sm.red[13][t - s]}));
      }
      if (t + s < T) {
        const M2<S> ga = mneg(mmul(RC, minv(get_m<S, T>(sm.red, 4, t + s))));
        nC = mmul(ga, get_m<S, T>(sm.red, 8, t + s));
        nB = madd(nB, mmul(ga, get_m<S, T>(sm.red, 0, t + s)));
        nd = vadd(nd, mvec(ga, V2<S>{sm.red[12][t + s], sm.red[13][t + s]}));
      }
    }
    RA = nA;
    RB = nB;
    RC = nC;
    Rd = nd;
    if constexpr (T != 32) __syncthreads();
  }
  const V2<S> St = mvec(minv(RB), Rd);
  x[0] = St;
  if constexpr (P >= 2) {
    // ---- 3. back-substitution with S_t and S_{t+1}
    V2<S> Sn = {S(0), S(0)};
    if constexpr (T == 32) {
      const V2<S> sd = shfl_down_v(St, 1);
      if (t + 1 < T) Sn = sd;
    } else {
      sm.sep[0][t] = St.x;
      sm.sep[1][t] = St.y;
      __syncthreads();
      if (t + 1 < T) Sn = {sm.sep[0][t + 1], sm.sep[1][t + 1]};
    }
    x[P - 1] = mvec(Binv[P - 1], vsub(vsub(dd[P - 1], mvec(Et[P - 1], St)), mvec(C[P - 1], Sn)));
#pragma unroll
    for (int l = P - 2; l >= 1; --l)
      x[l] = mvec(Binv[l], vsub(vsub(dd[l], mvec(Et[l], St)), mvec(C[l], x[l + 1])));
    if constexpr (T != 32) __syncthreads();
  }
}

// ---------------------------------------------------------------- CTA reductions (fixed order)

template <int T>
struct ReduceSmem {
  double v[T / 32];
  double w[T / 32];
};

template <int T>
__device__ __forceinline__ double cta_max(double v, ReduceSmem<T>& sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if constexpr (T == 32) return v;
  if ((threadIdx.x & 31) == 0) sm.v[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = sm.v[0];
#pragma unroll
  for (int i = 1; i < T / 32; ++i) r = fmax(r, sm.v[i]);
  __syncthreads();
  return r;
}

template <int T>
__device__ __forceinline__ float cta_max_f(float v, ReduceSmem<T>& sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if constexpr (T == 32) return v;
  if ((threadIdx.x & 31) == 0) sm.v[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = float(sm.v[0]);
#pragma unroll
  for (int i = 1; i < T / 32; ++i) r = fmaxf(r, float(sm.v[i]));
  __syncthreads();
  return r;
}

// Sum and max in one pass; the sum uses a fixed reduction tree (deterministic).
template <int T>
__device__ __forceinline__ void cta_sum_max(double& s, double& m, ReduceSmem<T>& sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if constexpr (T == 32) return;
  if ((threadIdx.x & 31) == 0) {
    sm.v[threadIdx.x >> 5] = s;
    sm.w[threadIdx.x >> 5] = m;
  }
  __syncthreads();
  double rs = sm.v[0], rm = sm.w[0];
#pragma unroll
  for (int i = 1; i < T / 32; ++i) {
    rs += sm.v[i];
    rm = fmax(rm, sm.w[i]);
  }
  __syncthreads();
  s = rs;
  m = rm;
}

}  // namespace chg
