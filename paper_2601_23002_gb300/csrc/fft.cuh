// Batched, strided mixed-radix FFTs in shared memory.
//
// Register codelets: radix 2, 3, 4, 5 written out; 6, 8, 9, 10, 12, 15, 16 by
// compile-time Cooley-Tukey composition of those, with twiddles folded into
// constants (trivial ones, 1 and +-i, become swaps/negations).
//
// Shared-memory passes: Stockham auto-sort (each radix-R pass reads R values
// n/R apart, twiddles them, applies the codelet and writes them Ns apart), out
// of place between two buffers so that no thread waits on another inside a
// pass.  Data element i of batch b sits at base + b*bs + i*es; threads are
// mapped batch-fastest, so batch-contiguous layouts (bs = 1) and row layouts
// with an odd row pitch are free of bank conflicts.
//
// Direction DIR = -1 computes X_k = sum_j x_j exp(-2 pi i jk/n) (forward),
// DIR = +1 the unnormalised inverse.
#pragma once
#include "common.cuh"

namespace ofdft {

// multiply by exp(DIR * 2 pi i K / N) with K, N compile-time
template <typename C, int N, int K, int DIR>
__device__ __forceinline__ C twiddle_c(C a) {
  constexpr int k = ((K % N) + N) % N;
  if constexpr (k == 0) {
    return a;
  } else if constexpr (2 * k == N) {
    a.x = -a.x; a.y = -a.y; return a;
  } else if constexpr (4 * k == N) {
    return DIR < 0 ? cmul_mi(a) : cmul_pi(a);
  } else if constexpr (4 * k == 3 * N) {
    return DIR < 0 ? cmul_pi(a) : cmul_mi(a);
  } else {
    using T = decltype(a.x);
    constexpr double c = cos2pi(k, N);
    constexpr double s = DIR * sin2pi(k, N);
    C w; w.x = (T)c; w.y = (T)s;
    return cmul(a, w);
  }
}

template <typename C, int R, int DIR> struct Codelet;

template <typename C, int DIR> struct Codelet<C, 1, DIR> {
  static __device__ __forceinline__ void run(C*) {}
};

template <typename C, int DIR> struct Codelet<C, 2, DIR> {
  static __device__ __forceinline__ void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  }
};

template <typename C, int DIR> struct Codelet<C, 3, DIR> {
  static __device__ __forceinline__ void run(C* v) {
    using T = decltype(v[0].x);
    const T h = (T)0.86602540378443864676372317075294;  // sin(2 pi/3)
    C t = cadd(v[1], v[2]);
    C a = v[0];
    a.x -= (T)0.5 * t.x; a.y -= (T)0.5 * t.y;
    C d = csub(v[1], v[2]);
    C b; b.x = h * d.x; b.y = h * d.y;
    v[0] = cadd(v[0], t);
    // X1 = a - i b (forward), X2 = a + i b
    C mib = cmul_mi(b);
    if constexpr (DIR < 0) { v[1] = cadd(a, mib); v[2] = csub(a, mib); }
    else { v[1] = csub(a, mib); v[2] = cadd(a, mib); }
  }
};

template <typename C, int DIR> struct Codelet<C, 4, DIR> {
  static __device__ __forceinline__ void run(C* v) {
    C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    C c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    v[0] = cadd(a, c); v[2] = csub(a, c);
    C mid = cmul_mi(d);   // -i d
    if constexpr (DIR < 0) { v[1] = cadd(b, mid); v[3] = csub(b, mid); }
    else { v[1] = csub(b, mid); v[3] = cadd(b, mid); }
  }
};

template <typename C, int DIR> struct Codelet<C, 5, DIR> {
  static __device__ __forceinline__ void run(C* v) {
    using T = decltype(v[0].x);
    const T c1 = (T)0.30901699437494742410229341718282;   // cos(2pi/5)
    const T c2 = (T)-0.80901699437494742410229341718282;  // cos(4pi/5)
    const T s1 = (T)0.95105651629515357211643933337938;   // sin(2pi/5)
    const T s2 = (T)0.58778525229247312916870595463907;   // sin(4pi/5)
    C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    C t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    C x0 = v[0];
    C a1, a2, b1, b2;
    a1.x = x0.x + c1 * t1.x + c2 * t2.x; a1.y = x0.y + c1 * t1.y + c2 * t2.y;
    a2.x = x0.x + c2 * t1.x + c1 * t2.x; a2.y = x0.y + c2 * t1.y + c1 * t2.y;
    b1.x = s1 * t3.x + s2 * t4.x; b1.y = s1 * t3.y + s2 * t4.y;
    b2.x = s2 * t3.x - s1 * t4.x; b2.y = s2 * t3.y - s1 * t4.y;
    v[0] = cadd(x0, cadd(t1, t2));
    C m1 = cmul_mi(b1), m2 = cmul_mi(b2);   // -i b
    if constexpr (DIR < 0) {
      v[1] = cadd(a1, m1); v[4] = csub(a1, m1); v[2] = cadd(a2, m2); v[3] = csub(a2, m2);
    } else {
      v[1] = csub(a1, m1); v[4] = cadd(a1, m1); v[2] = csub(a2, m2); v[3] = cadd(a2, m2);
    }
  }
};

// R = R1 * R2: x index j = R2 j1 + j2, output index k = k1 + R1 k2.
template <typename C, int R1, int R2, int DIR>
__device__ __forceinline__ void composite(C* v) {
  constexpr int R = R1 * R2;
  C t[R];
  static_for<0, R2>([&](auto J2) {
    constexpr int j2 = decltype(J2)::value;
    C u[R1];
    static_for<0, R1>([&](auto J1) { u[decltype(J1)::value] = v[R2 * decltype(J1)::value + j2]; });
    Codelet<C, R1, DIR>::run(u);
    static_for<0, R1>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      t[k1 * R2 + j2] = twiddle_c<C, R, j2 * k1, DIR>(u[k1]);
    });
  });
  static_for<0, R1>([&](auto K1) {
    constexpr int k1 = decltype(K1)::value;
    C u[R2];
    static_for<0, R2>([&](auto J2) { u[decltype(J2)::value] = t[k1 * R2 + decltype(J2)::value]; });
    Codelet<C, R2, DIR>::run(u);
    static_for<0, R2>([&](auto K2) { v[k1 + R1 * decltype(K2)::value] = u[decltype(K2)::value]; });
  });
}

#define OFDFT_COMPOSITE(R, R1, R2)                                                   \
  template <typename C, int DIR> struct Codelet<C, R, DIR> {                         \
    static __device__ __forceinline__ void run(C* v) { composite<C, R1, R2, DIR>(v); } \
  };
OFDFT_COMPOSITE(6, 2, 3)
OFDFT_COMPOSITE(8, 2, 4)
OFDFT_COMPOSITE(9, 3, 3)
OFDFT_COMPOSITE(10, 2, 5)
OFDFT_COMPOSITE(12, 3, 4)
OFDFT_COMPOSITE(15, 3, 5)
OFDFT_COMPOSITE(16, 4, 4)
#undef OFDFT_COMPOSITE

// ---------------------------------------------------------------------------
// Plan of one 1-D length: radices (product = n), at most 8 passes.
struct FftPlan1 {
  int n;
  int npass;
  int radix[8];
};

// Exact quotient a / d by one multiply-high: with M = ceil(2^32 / d),
// floor(a M / 2^32) = floor(a/d + e) where 0 <= e < a / 2^32, and a/d is at
// least 1/d below the next integer, so the result is exact whenever
// a d < 2^32 (here a < 2^17 and d < 2^10).  d = 1 gives M = 0 and is handled
// by the caller's select.  Integer division would cost about twenty
// instructions; a float reciprocal needs conversions, which GB300 issues on
// its narrow FP64 pipe.
__device__ __forceinline__ unsigned qmagic(unsigned d) { return d > 1 ? 0xFFFFFFFFu / d + 1u : 0u; }
__device__ __forceinline__ int qdiv(int a, unsigned d, unsigned M) {
  return d > 1 ? (int)__umulhi((unsigned)a, M) : a;
}

// One Stockham pass of radix R over nb transforms of length n.
// tw[t] = exp(-2 pi i t / n) for t in [0, n).
template <typename T, int R, int DIR>
__device__ __forceinline__ void stockham_pass(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out,
                                              int n, int Ns, int es, int bs, int nb,
                                              const cplx<T>* __restrict__ tw) {
  const int m = n / R;
  const int items = nb * m;
  const int step = n / (Ns * R);
  const unsigned Mnb = qmagic(nb), Mns = qmagic(Ns);
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int j = qdiv(it, nb, Mnb), b = it - j * nb;
    cplx<T> v[R];
    const cplx<T>* src = in + (size_t)b * bs;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * m) * es];
    const int jq = qdiv(j, Ns, Mns);
    const int k = j - jq * Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = tw[k * r * step];
        if (DIR > 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    Codelet<cplx<T>, R, DIR>::run(v);
    const int base = jq * Ns * R + k;
    cplx<T>* dst = out + (size_t)b * bs;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * Ns) * es] = v[r];
  }
}

// Full transform: data in buf[0]; returns the buffer holding the result.
// Both buffers use the same (es, bs) layout.  Ends with __syncthreads().
template <typename T, int DIR>
__device__ cplx<T>* fft_smem(cplx<T>* buf0, cplx<T>* buf1, const FftPlan1& p, int es, int bs, int nb,
                             const cplx<T>* __restrict__ tw) {
  cplx<T>* in = buf0;
  cplx<T>* out = buf1;
  int Ns = 1;
  for (int q = 0; q < p.npass; ++q) {
    const int R = p.radix[q];
    switch (R) {
      case 2: stockham_pass<T, 2, DIR>(in, out, p.n, Ns, es, bs, nb, tw); break;
      case 3: stockham_pass<T, 3, DIR>(in, out, p.n, Ns, es, bs, nb, tw); break;
      case 4: stockham_pass<T, 4, DIR>(in, out, p.n, Ns, es, bs, nb, tw); break;
      case 5: stockham_pass<T, 5, DIR>(in, out, p.n, Ns, es, bs, nb, tw); break;
      case 6: stockham_pass<T, 6, DIR>(in, out, p.n, Ns, es, bs, nb, tw); break;
      case 8: stockham_pass<T, 8, DIR>(in, out, p.n, Ns, es, bs, nb, tw); break;
      case 9: stockham_pass<T, 9, DIR>(in, out, p.n, Ns, es, bs, nb, tw); break;
      case 10: stockham_pass<T, 10, DIR>(in, out, p.n, Ns, es, bs, nb, tw); break;
      case 12: stockham_pass<T, 12, DIR>(in, out, p.n, Ns, es, bs, nb, tw); break;
      case 15: stockham_pass<T, 15, DIR>(in, out, p.n, Ns, es, bs, nb, tw); break;
      case 16: stockham_pass<T, 16, DIR>(in, out, p.n, Ns, es, bs, nb, tw); break;
      default: break;
    }
    __syncthreads();
    cplx<T>* t = in; in = out; out = t;
    Ns *= R;
  }
  return in;
}

}  // namespace ofdft
