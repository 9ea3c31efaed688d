// Register-resident line FFTs of compile-time length 2^k or 3 x 2^k, for the transform passes of
// the UNO preconditioner (Algorithm 2) on grids whose axes are 16..256 points long.
//
// A line of N = V * G complex values is held by G cooperating threads of one warp, V values
// each.  With n = g + G n1 (g < G, n1 < V) and k = k1 + V k2 (k1 < V, k2 < G),
//
//   X[k1 + V k2] = sum_g W_G^{g k2} W_N^{g k1} sum_n1 W_V^{n1 k1} x[g + G n1],
//
// so a line transform is a V-point DFT in every thread, a twiddle W_N^{g k1}, one exchange of
// values between the G threads through shared memory (synchronised by __syncwarp only), and
// V/G G-point DFTs per thread.  Two data distributions occur:
//   natural   : thread g holds v[n1] = x[g + G n1], n1 < V;
//   scattered : thread g holds v[j G + k2] = X[k1 + V k2] with k1 = g V/G + j (j < V/G).
// fft_dist_a maps natural to scattered, fft_dist_b scattered to natural (the same identity
// read from the other side).  Both take the direction DIR (-1 forward, +1 inverse; the
// transforms are unnormalized), so a forward transform followed by an inverse one needs no
// redistribution in between.
//
// Exchange scratch: the N complex slots of the line at scr[s * ss], s < N.  The value of
// (k1, t) lives in slot k1 G + ((t + k1 / (V/G)) mod G); the rotation spreads the accesses of a
// warp over the shared-memory banks for the lane layouts used by the kernels.
#pragma once
#include "fft.cuh"

namespace unocg {

// radix-16 DFT, natural order in and out: 4 x 4 with the inner twiddles W_16^(a b)
template <int DIR, typename C> __device__ __forceinline__ void dft16(C* v) {
  using T = decltype(v[0].x);
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;  // cos, sin(pi/8)
  const T h = (T)0.70710678118654752440;
  C y[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    C t[4] = {v[a], v[a + 4], v[a + 8], v[a + 12]};
    dft4<DIR>(t);
#pragma unroll
    for (int b = 0; b < 4; ++b) y[a][b] = t[b];
  }
  // y[a][b] *= W_16^(DIR a b) for a, b in 1..3; products a b in {1, 2, 3, 4, 6, 9}
  auto tw = [&](C x, int m) -> C {
    // W_16^m (forward, DIR < 0): cos(2 pi m / 16) - i sin(2 pi m / 16)
    T cr, si;
    switch (m) {
      case 1: cr = c1; si = s1; break;
      case 2: cr = h; si = h; break;
      case 3: cr = s1; si = c1; break;
      case 4: cr = (T)0; si = (T)1; break;
      case 6: cr = -h; si = h; break;
      default: cr = -c1; si = -s1; break;  // m = 9
    }
    const T sg = DIR < 0 ? -si : si;
    return mk<T>(x.x * cr - x.y * sg, x.x * sg + x.y * cr);
  };
#pragma unroll
  for (int a = 1; a < 4; ++a)
#pragma unroll
    for (int b = 1; b < 4; ++b) y[a][b] = tw(y[a][b], a * b);
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    C t[4] = {y[0][b], y[1][b], y[2][b], y[3][b]};
    dft4<DIR>(t);
#pragma unroll
    for (int c = 0; c < 4; ++c) v[b + 4 * c] = t[c];
  }
}

// cos(2 pi k / 24), k any integer (multiples of 15 degrees)
__host__ __device__ constexpr double cos24_q(int k) {  // 0 <= k <= 6
  return k == 0 ? 1.0 : k == 1 ? 0.96592582628906828675 : k == 2 ? 0.86602540378443864676
       : k == 3 ? 0.70710678118654752440 : k == 4 ? 0.5 : k == 5 ? 0.25881904510252076235 : 0.0;
}
__host__ __device__ constexpr double cos24(int k) {
  const int m = ((k % 24) + 24) % 24, r = m > 12 ? 24 - m : m;  // 0 <= r <= 12
  return r <= 6 ? cos24_q(r) : -cos24_q(12 - r);
}

// radix 3 M (M = 4, 8), natural order in and out: M-point DFTs of the samples a, a + 3, ...
// (a < 3), twiddles W_3M^(a b), 3-point DFTs across a.  With n = a + 3 m and k = b + M c:
//   X[b + M c] = sum_a W_3^(a c) W_3M^(a b) sum_m x[a + 3 m] W_M^(m b)
template <int DIR, int M, typename C> __device__ __forceinline__ void dft3m(C* v) {
  using T = decltype(v[0].x);
  constexpr int N = 3 * M, S = 24 / N;  // W_N^m = W_24^(S m)
  C y[3][M];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int m = 0; m < M; ++m) y[a][m] = v[a + 3 * m];
    if constexpr (M == 4) dft4<DIR>(y[a]);
    else dft8<DIR>(y[a]);
  }
#pragma unroll
  for (int a = 1; a < 3; ++a)
#pragma unroll
    for (int b = 1; b < M; ++b) {
      // W_N^(a b) = cos(2 pi a b / N) -/+ i sin(2 pi a b / N) (forward / inverse)
      const T cr = (T)cos24(S * a * b), si = (T)cos24(S * a * b - 6);
      const T sg = DIR < 0 ? -si : si;
      const C x = y[a][b];
      y[a][b] = mk<T>(x.x * cr - x.y * sg, x.x * sg + x.y * cr);
    }
#pragma unroll
  for (int b = 0; b < M; ++b) {
    C t[3] = {y[0][b], y[1][b], y[2][b]};
    dft3<DIR>(t);
#pragma unroll
    for (int c = 0; c < 3; ++c) v[b + M * c] = t[c];
  }
}

template <int R, int DIR, typename C> __device__ __forceinline__ void dft_pow2(C* v) {
  if constexpr (R == 2) dft2<DIR>(v);
  else if constexpr (R == 4) dft4<DIR>(v);
  else if constexpr (R == 8) dft8<DIR>(v);
  else if constexpr (R == 16) dft16<DIR>(v);
  else if constexpr (R == 12) dft3m<DIR, 4>(v);
  else if constexpr (R == 24) dft3m<DIR, 8>(v);
}

// split N = V * G with G a power of two, G | V, G <= 16, V <= 24 (V = 12, 24 for the axes of
// 3 x 2^k points)
template <int N> struct RegSplit;
template <> struct RegSplit<16> { static constexpr int V = 4, G = 4; };
template <> struct RegSplit<24> { static constexpr int V = 12, G = 2; };
template <> struct RegSplit<32> { static constexpr int V = 8, G = 4; };
template <> struct RegSplit<48> { static constexpr int V = 12, G = 4; };
template <> struct RegSplit<64> { static constexpr int V = 8, G = 8; };
template <> struct RegSplit<96> { static constexpr int V = 24, G = 4; };
template <> struct RegSplit<128> { static constexpr int V = 16, G = 8; };
template <> struct RegSplit<192> { static constexpr int V = 24, G = 8; };
template <> struct RegSplit<256> { static constexpr int V = 16, G = 16; };

// threads per line of the split of n (0: no register split for n), for host-side grid sizes
__host__ __device__ constexpr int reg_split_g(int n) {
  return n == 16 ? 4 : n == 24 ? 2 : n == 32 ? 4 : n == 48 ? 4 : n == 64 ? 8 : n == 96 ? 4 : n == 128 ? 8
       : n == 192 ? 8 : n == 256 ? 16 : 0;
}

template <int N> __device__ __forceinline__ int reg_slot(int k1, int t) {
  constexpr int V = RegSplit<N>::V, G = RegSplit<N>::G, VG = V / G;
  return k1 * G + ((t + k1 / VG) & (G - 1));
}

// x * W^(DIR m) with W the forward root stored in the table
template <int DIR, typename C> __device__ __forceinline__ C twiddle(C x, C w) {
  if (DIR > 0) w.y = -w.y;
  return cmul(x, w);
}

// natural -> scattered (see the header).  slot(s) is this line's exchange slot s < N (a reference
// into shared memory); tw: W_N^m.  All lanes of the warp must call it; the slots may be reused
// after the caller's next __syncwarp().
template <int N, int DIR, typename C, typename Slot>
__device__ __forceinline__ void fft_dist_a_at(C* v, int g, Slot slot, const C* __restrict__ tw) {
  constexpr int V = RegSplit<N>::V, G = RegSplit<N>::G, VG = V / G;
  dft_pow2<V, DIR>(v);
#pragma unroll
  for (int k1 = 1; k1 < V; ++k1) v[k1] = twiddle<DIR>(v[k1], tw[g * k1]);
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < V; ++k1) slot(reg_slot<N>(k1, g)) = v[k1];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < VG; ++j)
#pragma unroll
    for (int t = 0; t < G; ++t) v[j * G + t] = slot(reg_slot<N>(g * VG + j, t));
#pragma unroll
  for (int j = 0; j < VG; ++j) dft_pow2<G, DIR>(v + j * G);
}

// scattered -> natural
template <int N, int DIR, typename C, typename Slot>
__device__ __forceinline__ void fft_dist_b_at(C* v, int g, Slot slot, const C* __restrict__ tw) {
  constexpr int V = RegSplit<N>::V, G = RegSplit<N>::G, VG = V / G;
#pragma unroll
  for (int j = 0; j < VG; ++j) dft_pow2<G, DIR>(v + j * G);
#pragma unroll
  for (int j = 0; j < VG; ++j)
#pragma unroll
    for (int t = 1; t < G; ++t) v[j * G + t] = twiddle<DIR>(v[j * G + t], tw[t * (g * VG + j)]);
  __syncwarp();
#pragma unroll
  for (int j = 0; j < VG; ++j)
#pragma unroll
    for (int t = 0; t < G; ++t) slot(reg_slot<N>(g * VG + j, t)) = v[j * G + t];
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < V; ++k1) v[k1] = slot(reg_slot<N>(k1, g));
  dft_pow2<V, DIR>(v);
}

// the slots at base[s ^ x]: a line's own N slots with the slot index bits of x flipped (two lines
// whose accesses would fall on the same banks use complementary banks with x = 0 and x = 8)
template <typename C> struct XorSlot {
  C* base;
  int x;
  __device__ __forceinline__ C& operator()(int s) const { return base[s ^ x]; }
};
// the slots at scr[s * ss]
template <typename C> struct StrideSlot {
  C* scr;
  int ss;
  __device__ __forceinline__ C& operator()(int s) const { return scr[s * ss]; }
};
template <int N, int DIR, typename C>
__device__ __forceinline__ void fft_dist_a(C* v, int g, C* scr, int ss, const C* __restrict__ tw) {
  fft_dist_a_at<N, DIR>(v, g, StrideSlot<C>{scr, ss}, tw);
}
template <int N, int DIR, typename C>
__device__ __forceinline__ void fft_dist_b(C* v, int g, C* scr, int ss, const C* __restrict__ tw) {
  fft_dist_b_at<N, DIR>(v, g, StrideSlot<C>{scr, ss}, tw);
}

// index k of value v[j G + k2] in the scattered distribution of thread g
template <int N> __device__ __forceinline__ int scat_index(int g, int j, int k2) {
  constexpr int V = RegSplit<N>::V, G = RegSplit<N>::G, VG = V / G;
  return g * VG + j + V * k2;
}

// ---------------------------------------------------------------- real-to-complex rows
// shared by the plane passes (k_fft_reg.cu, k_plane_cl.cu)
template <typename T>
__device__ __forceinline__ void load_tw_reg(cplx<T>* dst, const void* src, int N) {
  const cplx<T>* s = (const cplx<T>*)src;
  for (int i = threadIdx.x; i < N; i += blockDim.x) dst[i] = s[i];
}

// X(k), X(Nh-k) from the half-length spectrum Z in one row (in place), pair k <= Nh/2
template <typename T>
__device__ __forceinline__ void r2c_pair(cplx<T>* b, int k, int Nh, const cplx<T>* __restrict__ twN) {
  using C = cplx<T>;
  const T half = (T)0.5;
  if (k == 0) {
    C z = b[0];
    b[0] = mk<T>(z.x + z.y, (T)0);
    b[Nh] = mk<T>(z.x - z.y, (T)0);
    return;
  }
  const int k2 = Nh - k;
  C zk = b[k], zm = b[k2];
  C e = mk<T>(half * (zk.x + zm.x), half * (zk.y - zm.y));
  C o = mk<T>(half * (zk.y + zm.y), -half * (zk.x - zm.x));
  C xk = cadd(e, cmul(twN[k], o));
  if (k2 != k) {
    C e2 = mk<T>(half * (zm.x + zk.x), half * (zm.y - zk.y));
    C o2 = mk<T>(half * (zm.y + zk.y), -half * (zm.x - zk.x));
    b[k2] = cadd(e2, cmul(twN[k2], o2));
  }
  b[k] = xk;
}

// inverse of r2c_pair up to the factor of the unnormalized inverse (see c2r_pre)
template <typename T>
__device__ __forceinline__ void c2r_pair(cplx<T>* b, int k, int Nh, const cplx<T>* __restrict__ twN) {
  using C = cplx<T>;
  if (k == 0) {
    T x0 = b[0].x, xn = b[Nh].x;
    b[0] = mk<T>(x0 + xn, x0 - xn);
    return;
  }
  const int k2 = Nh - k;
  C xk = b[k], xm = b[k2];
  C wk = twN[k];
  wk.y = -wk.y;
  C e = mk<T>(xk.x + xm.x, xk.y - xm.y);
  C o = cmul(mk<T>(xk.x - xm.x, xk.y + xm.y), wk);
  C zk = mk<T>(e.x - o.y, e.y + o.x);
  if (k2 != k) {
    C w2 = twN[k2];
    w2.y = -w2.y;
    C e2 = mk<T>(xm.x + xk.x, xm.y - xk.y);
    C o2 = cmul(mk<T>(xm.x - xk.x, xm.y + xk.y), w2);
    b[k2] = mk<T>(e2.x - o2.y, e2.y + o2.x);
  }
  b[k] = zk;
}


}  // namespace unocg
