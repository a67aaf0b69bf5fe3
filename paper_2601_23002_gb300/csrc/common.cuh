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

// Asynchronous global -> shared copies (cp.async).  pred == false copies no
// bytes and zero-fills the destination (the source pointer must still be a
// valid address).  Copies of one thread complete in commit-group order.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, bool pred) {
  static_assert(B == 4 || B == 8 || B == 16, "cp.async size");
  const int src = pred ? B : 0;
  if constexpr (B == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src)
                 : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(smem)), "l"(gmem), "n"(B),
                 "r"(src)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// copy one complex element (8 or 16 bytes)
template <typename C> __device__ __forceinline__ void cp_async_c(C* smem, const C* gmem, bool pred) {
  cp_async<sizeof(C)>(smem, gmem, pred);
}

// Per-thread accumulators.  FP64 plans add in double.  FP32 plans add in
// float with Kahan compensation (GB300 issues FP64 at 1/58 of the FP32 rate,
// so per-element FP64 adds would dominate an FP32 kernel); the compensated
// float sum of a thread's few dozen terms is then combined across the block
// and grid in double.
template <typename T> struct Acc;
template <> struct Acc<double> {
  double s = 0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<float> {
  float s = 0, c = 0;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// Block sums of per-thread accumulators, written by thread 0 to out[].
// For float accumulators the warp-level part runs in compensated float-float
// arithmetic (a (hi, lo) pair per value, combined with Knuth's TwoSum) and
// only the per-warp results are converted to double: on GB300 a handful of
// FP64 operations per thread already cost as much as a streaming kernel.
struct FF { float hi, lo; };
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  const float lo = a.lo + b.lo + e;
  const float h2 = s + lo;
  return FF{h2, lo - (h2 - s)};
}
__device__ __forceinline__ FF ff_from(const Acc<float>& a) {
  const float hi = a.s - a.c;
  return FF{hi, (a.s - hi) - a.c};
}

template <int NQ>
__device__ __forceinline__ void block_sum_acc(Acc<double> (&a)[NQ], double* scratch, double* out) {
  double v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = a[q].get();
  block_sum<NQ>(v, scratch, out);
}

template <int NQ>
__device__ __forceinline__ void block_sum_acc(Acc<float> (&a)[NQ], double* scratch, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    FF f = ff_from(a[q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      FF g;
      g.hi = __shfl_xor_sync(0xffffffffu, f.hi, o);
      g.lo = __shfl_xor_sync(0xffffffffu, f.lo, o);
      f = ff_add(f, g);
    }
    if (lane == 0) scratch[q * 32 + wid] = (double)f.hi + (double)f.lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < NQ; ++q) {
      double t = 0;
      for (int w = 0; w < nw; ++w) t += scratch[q * 32 + w];
      out[q] = t;
    }
  }
  __syncthreads();
}

// Short per-thread sums (a thread adds at most a few dozen terms): plain
// accumulation in the plan's precision, converted to the compensated form
// for the block reduction.
template <typename T> struct AccShort {
  T s = 0;
  __device__ __forceinline__ void add(T x) { s += x; }
};
template <int NQ, typename T>
__device__ __forceinline__ void block_sum_short(AccShort<T> (&a)[NQ], double* scratch, double* out) {
  Acc<T> b[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) { b[q].s = a[q].s; if constexpr (sizeof(T) == 4) b[q].c = 0; }
  block_sum_acc<NQ>(b, scratch, out);
}

// Block sums through a shared-memory tree.  Reducing one value per lane with
// warp shuffles redoes every addition on all 32 lanes (5 levels x 32 lanes
// for 31 useful additions); with many per-thread sums that tail costs as much
// as a streaming kernel's main loop.  Here each thread parks its nq values in
// column q of a scratch array (row pitch blockDim + 1 against bank
// conflicts), and the block adds pairs h apart, h = blockDim/2, ..., 1, every
// thread taking a share of all columns' pairs.  Floats are carried as
// (hi, lo) pairs added with TwoSum, so the tree adds no rounding error of
// float order; the order is fixed, so results are deterministic.
// blockDim must be a power of two; scratch holds nq * (blockDim + 1) values of
// the scratch type (float2 / double).  dst[q] (global or shared) is written by
// thread q < nq; the function begins and ends with a block barrier.
template <typename T> struct TreeVal;
template <> struct TreeVal<float> { using type = float2; };
template <> struct TreeVal<double> { using type = double; };

__device__ __forceinline__ float2 tree_add(float2 a, float2 b) {
  const FF r = ff_add(FF{a.x, a.y}, FF{b.x, b.y});
  return make_float2(r.hi, r.lo);
}
__device__ __forceinline__ double tree_add(double a, double b) { return a + b; }
__device__ __forceinline__ double tree_get(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ double tree_get(double a) { return a; }
__device__ __forceinline__ float2 tree_put(const Acc<float>& a) {
  const FF f = ff_from(a);
  return make_float2(f.hi, f.lo);
}
__device__ __forceinline__ double tree_put(const Acc<double>& a) { return a.get(); }

// Tree over values already parked in scr (column q at scr + q * (blockDim + 1));
// afterwards column q's sum sits in scr[q * (blockDim + 1)].
template <typename V>
__device__ __forceinline__ void block_tree_core(int nq, V* scr) {
  const int nt = blockDim.x, pitch = nt + 1, t = threadIdx.x;
  __syncthreads();
  for (int h = nt >> 1, lg = __ffs(nt) - 2; h >= 1; h >>= 1, --lg) {
    for (int w = t; w < nq * h; w += nt) {
      const int q = w >> lg, i = w & (h - 1);
      V* c = scr + q * pitch;
      c[i] = tree_add(c[i], c[i + h]);
    }
    __syncthreads();
  }
}

// Sums of per-thread accumulators a[0..nq) over the block; thread q < nq
// writes column q's sum to dst[q] as a double.
template <int NQMAX, typename T>
__device__ __forceinline__ void block_sum_tree(const Acc<T>* a, int nq, double* dst,
                                               typename TreeVal<T>::type* scr) {
  const int pitch = blockDim.x + 1, t = threadIdx.x;
  __syncthreads();                                   // scratch may alias data still being read
#pragma unroll
  for (int q = 0; q < NQMAX; ++q)
    if (q < nq) scr[q * pitch + t] = tree_put(a[q]);
  block_tree_core(nq, scr);
  if (t < nq) dst[t] = tree_get(scr[t * pitch]);
  __syncthreads();
}
template <int NQ, typename T>
__device__ __forceinline__ void block_sum_tree(const AccShort<T> (&a)[NQ], double* dst,
                                               typename TreeVal<T>::type* scr) {
  Acc<T> b[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) { b[q].s = a[q].s; if constexpr (sizeof(T) == 4) b[q].c = 0; }
  block_sum_tree<NQ, T>(b, NQ, dst, scr);
}
// As above, but the sums stay in tree form (float-float pairs for float,
// doubles for double): dst[q] = column q's sum.  Partial sums that a later
// pass adds up stay on the FP32 pipe this way.
template <int NQ, typename T>
__device__ __forceinline__ void block_sum_tree_raw(const AccShort<T> (&a)[NQ], typename TreeVal<T>::type* dst,
                                                   typename TreeVal<T>::type* scr) {
  const int pitch = blockDim.x + 1, t = threadIdx.x;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    Acc<T> b;
    b.s = a[q].s;
    if constexpr (sizeof(T) == 4) b.c = 0;
    scr[q * pitch + t] = tree_put(b);
  }
  block_tree_core(NQ, scr);
  if (t < NQ) dst[t] = scr[t * pitch];
  __syncthreads();
}
template <typename T>
__host__ __device__ constexpr size_t tree_scratch_bytes(int nq, int nt) {
  return (size_t)nq * (nt + 1) * 8;   // float2 or double
}

// True in exactly one block: the last to arrive.  Every block must call it
// (after its thread 0 has written the block's partial results); the last one
// then reads all partials (use __ldcg) and resets the counter for the next
// launch in the stream.
__device__ __forceinline__ bool arrive_last(unsigned int* counter) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// One block: out[c] = sum_r partial[r * cols + c], fixed order, FP64.  Thread
// t sums column t % cols over rows t / cols, t / cols + k, ... (k = blockDim /
// cols row groups, loads coalesced along each row); then one thread per column
// adds the k group sums.  Requires cols <= blockDim.x.
__device__ __forceinline__ void block_sum_columns(const double* partial, int rows, int cols, double* out,
                                                  double* /*unused*/) {
  __shared__ double colscr[1024];
  // k = the largest power of two with k * cols <= blockDim.x threads per column
  int k = 1;
  while (2 * k * cols <= (int)blockDim.x) k *= 2;
  const int t = threadIdx.x;
  const int c = t % cols, g = t / cols;
  double v = 0;
  if (g < k) {
    // eight rows' loads in flight at a time, added in row order
    int r = g;
    for (; r + 7 * k < rows; r += 8 * k) {
      double x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = __ldcg(partial + (size_t)(r + u * k) * cols + c);
#pragma unroll
      for (int u = 0; u < 8; ++u) v += x[u];
    }
    for (; r < rows; r += k) v += __ldcg(partial + (size_t)r * cols + c);
    colscr[g * cols + c] = v;
  }
  __syncthreads();
  // pairwise tree over the k group sums of each column (fixed order): log2(k)
  // dependent FP64 additions instead of k
  for (int h = k / 2; h >= 1; h /= 2) {
    if (g < h) colscr[g * cols + c] += colscr[(g + h) * cols + c];
    __syncthreads();
  }
  if (t < cols) out[t] = colscr[t];
  __syncthreads();
}

// Block-wide sums of nq <= NQMAX per-thread accumulators in one pass: each
// warp reduces every value (float-float for float accumulators), lane 0 parks
// it in shared memory, then thread q < nq adds the warp results in double and
// writes dst[q] (deterministic).
// wres: shared scratch of 32 * NQMAX doubles.
template <int NQMAX, typename T>
__device__ __forceinline__ void block_sum_many(const Acc<T>* a, int nq, double* dst, double* wres) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NQMAX; ++q) {
    if (q < nq) {
      double r;
      if constexpr (sizeof(T) == 4) {
        FF f = ff_from(a[q]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          FF g;
          g.hi = __shfl_xor_sync(0xffffffffu, f.hi, o);
          g.lo = __shfl_xor_sync(0xffffffffu, f.lo, o);
          f = ff_add(f, g);
        }
        r = (double)f.hi + (double)f.lo;
      } else {
        r = warp_sum(a[q].get());
      }
      if (lane == 0) wres[wid * NQMAX + q] = r;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < nq) {
    double s = 0;
    for (int w = 0; w < nw; ++w) s += wres[w * NQMAX + threadIdx.x];
    dst[threadIdx.x] = s;
  }
  __syncthreads();
}

}  // namespace ofdft
