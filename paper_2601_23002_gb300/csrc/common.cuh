// Common device types and helpers for the OFDFT kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>

namespace ofdft {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T x, T y) {
  cplx<T> c; c.x = x; c.y = y; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) { a.x *= s; a.y *= s; return a; }
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// multiply by -i and +i
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }
template <typename C> __device__ __forceinline__ C cmul_pi(C a) { C r; r.x = -a.y; r.y = a.x; return r; }

// ---------------------------------------------------------------------------
// Compile-time cos/sin of 2*pi*k/n for the register codelets: exact integer
// octant reduction, then Taylor series on [0, pi/4] (error below 1e-17).
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double taylor_sin(double x) {
  double x2 = x * x, t = x, s = x;
  for (int k = 1; k < 14; ++k) { t *= -x2 / ((2.0 * k) * (2.0 * k + 1.0)); s += t; }
  return s;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double x2 = x * x, t = 1.0, s = 1.0;
  for (int k = 1; k < 14; ++k) { t *= -x2 / ((2.0 * k - 1.0) * (2.0 * k)); s += t; }
  return s;
}
// cos(2 pi k / n) and sin(2 pi k / n) for integers
__host__ __device__ constexpr double cos2pi(long k, long n) {
  long a = ((k % n) + n) % n;           // angle 2 pi a / n in [0, 2 pi)
  long q = (4 * a) / n;                 // quadrant
  long r = 4 * a - q * n;               // angle within quadrant = (pi/2) r / n
  // cos over the quadrant: q=0: cos(x); q=1: -sin(x); q=2: -cos(x); q=3: sin(x)
  double x = 0.5 * kPi * (double)r / (double)n;
  bool swap = 2 * r > n;                // use complement to stay in [0, pi/4]
  double xc = 0.5 * kPi * (double)(n - r) / (double)n;
  double c = swap ? taylor_sin(xc) : taylor_cos(x);
  double s = swap ? taylor_cos(xc) : taylor_sin(x);
  return q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
}
__host__ __device__ constexpr double sin2pi(long k, long n) { return cos2pi(4 * k - n, 4 * n); }  // sin t = cos(t - pi/2)

template <int B, int E, typename F> __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// FP64 block reduction helpers -------------------------------------------------
static __device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum NQ per-thread values over the block; thread 0 gets the totals in out[].
// scratch: shared double[NQ * 32].
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double* scratch, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double s = warp_sum(v[q]);
    if (lane == 0) scratch[q * 32 + wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = lane < nw ? scratch[q * 32 + lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) out[q] = s;
    }
  }
  __syncthreads();
}

}  // namespace ofdft
