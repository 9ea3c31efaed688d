// Shared-memory FFT engine for the unitary transform of the UNO preconditioner.
//
// Batches of lines held in shared memory are transformed with a mixed-radix Stockham
// autosort (radix 2, 3, 4, 5; natural order in and out), ping-ponging between two buffers
// of the same layout, one butterfly per thread at a time.  Transforms are unnormalized: forward uses
// W = exp(-2 pi i / N), inverse exp(+2 pi i / N); the 1/n of the unitary pair is applied
// once in the frequency-domain block multiply.
//
// Real rows of even length N are transformed through the half-length complex transform of
// z[m] = x[2m] + i x[2m+1] followed by the standard split into even/odd spectra.
#pragma once
#include "common.cuh"

namespace unocg {

// ---------------------------------------------------------------- small DFT kernels
template <int DIR, typename C> __device__ __forceinline__ void dft2(C* v) {
  C a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <int DIR, typename C> __device__ __forceinline__ void dft3(C* v) {
  using T = decltype(v[0].x);
  const T h = (T)0.5, s3 = (T)0.86602540378443864676;  // sin(2 pi / 3)
  C s = cadd(v[1], v[2]);
  C d = csub(v[1], v[2]);
  C a = v[0];
  v[0] = cadd(a, s);
  C t = mk<T>(a.x - h * s.x, a.y - h * s.y);
  C b = mk<T>(s3 * d.x, s3 * d.y);
  C mib = cmul_mi<DIR>(b);  // -i b (forward)
  v[1] = cadd(t, mib);
  v[2] = csub(t, mib);
}

template <int DIR, typename C> __device__ __forceinline__ void dft4(C* v) {
  C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  C c = cadd(v[1], v[3]), d = cmul_mi<DIR>(csub(v[1], v[3]));
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}

template <int DIR, typename C> __device__ __forceinline__ void dft5(C* v) {
  using T = decltype(v[0].x);
  const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
  const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;   // sin(2pi/5), sin(4pi/5)
  C x0 = v[0];
  C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  C t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  C a1 = mk<T>(x0.x + c1 * t1.x + c2 * t2.x, x0.y + c1 * t1.y + c2 * t2.y);
  C a2 = mk<T>(x0.x + c2 * t1.x + c1 * t2.x, x0.y + c2 * t1.y + c1 * t2.y);
  C b1 = mk<T>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
  C b2 = mk<T>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
  C m1 = cmul_mi<DIR>(b1), m2 = cmul_mi<DIR>(b2);
  v[0] = cadd(x0, cadd(t1, t2));
  v[1] = cadd(a1, m1);
  v[4] = csub(a1, m1);
  v[2] = cadd(a2, m2);
  v[3] = csub(a2, m2);
}

// radix 8 = two radix-4 DFTs of the even and odd samples, combined with W_8^k
template <int DIR, typename C> __device__ __forceinline__ void dft8(C* v) {
  using T = decltype(v[0].x);
  const T s = (T)0.70710678118654752440;
  C a[4] = {v[0], v[2], v[4], v[6]};
  C b[4] = {v[1], v[3], v[5], v[7]};
  dft4<DIR>(a);
  dft4<DIR>(b);
  // W_8^1 = (1 - i)/sqrt2 (forward), W_8^2 = -i, W_8^3 = (-1 - i)/sqrt2
  C b1 = mk<T>(s * (b[1].x + b[1].y), s * (b[1].y - b[1].x));
  if (DIR > 0) b1 = mk<T>(s * (b[1].x - b[1].y), s * (b[1].y + b[1].x));
  C b2 = cmul_mi<DIR>(b[2]);
  C b3 = mk<T>(s * (-b[3].x + b[3].y), s * (-b[3].y - b[3].x));
  if (DIR > 0) b3 = mk<T>(s * (-b[3].x - b[3].y), s * (-b[3].y + b[3].x));
  v[0] = cadd(a[0], b[0]);
  v[4] = csub(a[0], b[0]);
  v[1] = cadd(a[1], b1);
  v[5] = csub(a[1], b1);
  v[2] = cadd(a[2], b2);
  v[6] = csub(a[2], b2);
  v[3] = cadd(a[3], b3);
  v[7] = csub(a[3], b3);
}

template <int DIR, int R, typename C> __device__ __forceinline__ void dftR(C* v) {
  if (R == 2) dft2<DIR>(v);
  else if (R == 3) dft3<DIR>(v);
  else if (R == 4) dft4<DIR>(v);
  else if (R == 5) dft5<DIR>(v);
  else dft8<DIR>(v);
}

// floor(x / d) for 0 <= x < 2^20 and 1 <= d <= 2^12 by an integer multiply-high with
// m = floor(2^32 / d) + 1 (exact there: x (m d - 2^32) < 2^32); m = 0 encodes d = 1.
struct UDiv {
  unsigned m;
};
__device__ __forceinline__ UDiv udiv_of(int d) {
  UDiv u;
  u.m = d > 1 ? (unsigned)(0xFFFFFFFFu / (unsigned)d) + 1u : 0u;
  return u;
}
__device__ __forceinline__ int udiv(int x, UDiv u) { return u.m ? (int)__umulhi((unsigned)x, u.m) : x; }

// ---------------------------------------------------------------- one Stockham stage
// Lines: element (line, idx) at buf[line*ls + idx*es].  Work item = (line, j), j < N/R, with
// the line index fastest across threads (conflict-free for both row and column layouts).
// Out of place: reads src, writes dst.  `tw` holds W_N^m, m < N (shared memory).
template <typename T, int DIR, int R>
__device__ __forceinline__ void fft_stage(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst,
                                          int nlines, int ls, int es, int N, int Ns,
                                          const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  const int NR = N / R;
  const int total = nlines * NR;
  const int stride = N / (Ns * R);
  const UDiv rl = udiv_of(nlines), rs = udiv_of(Ns);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int j = udiv(idx, rl);
    const int line = idx - j * nlines;
    const C* b = src + line * ls;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = b[(j + r * NR) * es];
    const int q = udiv(j, rs);
    const int k = j - q * Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = tw[r * k * stride];
        if (DIR > 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    dftR<DIR, R>(v);
    const int base = q * Ns * R + k;
    C* o = dst + line * ls;
#pragma unroll
    for (int r = 0; r < R; ++r) o[(base + r * Ns) * es] = v[r];
  }
  __syncthreads();
}

// Transform `nlines` lines of length pl.N held in `a` (same layout in the scratch buffer `b`).
// Returns the buffer that holds the result (a after an even number of stages, else b).
template <typename T, int DIR>
__device__ cplx<T>* fft_lines(cplx<T>* a, cplx<T>* b, int nlines, int ls, int es, const FftPlan& pl,
                              const cplx<T>* __restrict__ tw) {
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.radix[s];
    switch (R) {
      case 2: fft_stage<T, DIR, 2>(a, b, nlines, ls, es, pl.N, Ns, tw); break;
      case 3: fft_stage<T, DIR, 3>(a, b, nlines, ls, es, pl.N, Ns, tw); break;
      case 4: fft_stage<T, DIR, 4>(a, b, nlines, ls, es, pl.N, Ns, tw); break;
      case 5: fft_stage<T, DIR, 5>(a, b, nlines, ls, es, pl.N, Ns, tw); break;
      default: fft_stage<T, DIR, 8>(a, b, nlines, ls, es, pl.N, Ns, tw); break;
    }
    Ns *= R;
    cplx<T>* t = a;
    a = b;
    b = t;
  }
  return a;
}

// Copy a twiddle table W_N^m (m < N) from global to shared memory.
template <typename T>
__device__ __forceinline__ void load_tw(cplx<T>* dst, const void* src, int N) {
  const cplx<T>* s = (const cplx<T>*)src;
  for (int i = threadIdx.x; i < N; i += blockDim.x) dst[i] = s[i];
}

// ---------------------------------------------------------------- real <-> half-complex rows
// After the forward half-length transform of z[m] = x[2m] + i x[2m+1] (Nh = N/2 values in
// slots 0..Nh-1 of each row), produce X(k), k = 0..Nh, in slots 0..Nh:
//   X(k) = (Z(k) + conj Z(Nh-k))/2 - (i/2) W_N^k (Z(k) - conj Z(Nh-k)),  Z(Nh) = Z(0).
template <typename T>
__device__ void r2c_post(cplx<T>* buf, int nrows, int P, int Nh, const cplx<T>* __restrict__ twN) {
  using C = cplx<T>;
  const int npairs = Nh / 2 + 1;
  const T half = (T)0.5;
  const UDiv rr = udiv_of(nrows);
  for (int idx = threadIdx.x; idx < nrows * npairs; idx += blockDim.x) {
    const int k = udiv(idx, rr), row = idx - k * nrows;
    C* b = buf + row * P;
    if (k == 0) {
      C z = b[0];
      b[0] = mk<T>(z.x + z.y, (T)0);
      b[Nh] = mk<T>(z.x - z.y, (T)0);
    } else {
      int k2 = Nh - k;
      C zk = b[k], zm = b[k2];
      // X(k)
      C e = mk<T>(half * (zk.x + zm.x), half * (zk.y - zm.y));        // (Zk + conj Zm)/2
      C o = mk<T>(half * (zk.y + zm.y), -half * (zk.x - zm.x));       // -(i/2)(Zk - conj Zm)
      C xk = cadd(e, cmul(twN[k], o));
      if (k2 != k) {
        C e2 = mk<T>(half * (zm.x + zk.x), half * (zm.y - zk.y));
        C o2 = mk<T>(half * (zm.y + zk.y), -half * (zm.x - zk.x));
        b[k2] = cadd(e2, cmul(twN[k2], o2));
      }
      b[k] = xk;
    }
  }
  __syncthreads();
}

// Inverse of r2c_post up to the factor that makes the following unnormalized half-length
// inverse transform return y = G_N X (the unnormalized inverse DFT of the Hermitian row):
//   Z(k) = E(k) + i O(k),  E(k) = X(k) + conj X(Nh-k),  O(k) = (X(k) - conj X(Nh-k)) W_N^{-k}.
// The imaginary parts of X(0) and X(Nh) are ignored (they vanish for Hermitian data).
template <typename T>
__device__ void c2r_pre(cplx<T>* buf, int nrows, int P, int Nh, const cplx<T>* __restrict__ twN) {
  using C = cplx<T>;
  const int npairs = Nh / 2 + 1;
  const UDiv rr = udiv_of(nrows);
  for (int idx = threadIdx.x; idx < nrows * npairs; idx += blockDim.x) {
    const int k = udiv(idx, rr), row = idx - k * nrows;
    C* b = buf + row * P;
    if (k == 0) {
      T x0 = b[0].x, xn = b[Nh].x;
      b[0] = mk<T>(x0 + xn, x0 - xn);
    } else {
      int k2 = Nh - k;
      C xk = b[k], xm = b[k2];
      C wk = twN[k];
      wk.y = -wk.y;
      C e = mk<T>(xk.x + xm.x, xk.y - xm.y);
      C o = cmul(mk<T>(xk.x - xm.x, xk.y + xm.y), wk);
      C zk = mk<T>(e.x - o.y, e.y + o.x);  // E + i O
      if (k2 != k) {
        C w2 = twN[k2];
        w2.y = -w2.y;
        C e2 = mk<T>(xm.x + xk.x, xm.y - xk.y);
        C o2 = cmul(mk<T>(xm.x - xk.x, xm.y + xk.y), w2);
        b[k2] = mk<T>(e2.x - o2.y, e2.y + o2.x);
      }
      b[k] = zk;
    }
  }
  __syncthreads();
}

}  // namespace unocg
