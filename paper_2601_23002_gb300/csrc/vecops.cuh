// Grid-vector kernels of the minimiser: fused multi-dot products, linear
// combinations and the L-BFGS accept step.  FP64 accumulation throughout.
#pragma once
#include "common.cuh"

namespace ofdft {

constexpr int kMaxV = 9;    // vectors per gram launch (longer lists are chunked)
constexpr int kMaxW = 4;    // targets per gram launch
constexpr int kMaxLin = 20; // terms of a linear combination (1 + 2 m, m <= 8)

// 16-byte vector loads and stores of a real array (4 floats or 2 doubles).
template <typename T> struct V16;
template <> struct V16<float> { using type = float4; static constexpr int K = 4; };
template <> struct V16<double> { using type = double2; static constexpr int K = 2; };
template <typename T>
__device__ __forceinline__ void ld16(const T* p, size_t i, T (&o)[V16<T>::K]) {
  const typename V16<T>::type v = reinterpret_cast<const typename V16<T>::type*>(p)[i];
  static_assert(sizeof(v) == sizeof(o), "vector size");
  memcpy(o, &v, sizeof(o));
}
template <typename T>
__device__ __forceinline__ void st16(T* p, size_t i, const T (&o)[V16<T>::K]) {
  typename V16<T>::type v;
  memcpy(&v, o, sizeof(o));
  reinterpret_cast<typename V16<T>::type*>(p)[i] = v;
}

template <typename T> struct VecList {
  const T* v[kMaxLin];
  double c[kMaxLin];
  int nv;
};

template <typename T>
__global__ void k_fill(T* __restrict__ x, T v, size_t N) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    x[i] = v;
}

template <typename T>
__global__ void k_sqrt_clamp(T* __restrict__ psi, const T* __restrict__ rho, size_t N) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    psi[i] = sqrt(fmax(rho[i], (T)0));
}

// rho = scale * psi^2
template <typename T>
__global__ void k_density(T* __restrict__ rho, const T* __restrict__ psi, double scale, size_t N) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const T p = psi[i];
    rho[i] = (T)scale * p * p;
  }
}

// g = 2 scale (gp - mu psi)
template <typename T>
__global__ void k_project(T* __restrict__ g, const T* __restrict__ gp, const T* __restrict__ psi, double scale,
                          double mu, size_t N) {
  const T a = (T)(2.0 * scale), m = (T)mu;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    g[i] = a * (gp[i] - m * psi[i]);
}

// All dot products <V_i, W_j>, i < nv <= kMaxV, j < NW.  Per block into
// partial[block][i*NW + j]; the last block sums the columns into out[] in a
// fixed order.  Products and per-thread sums in the vectors' precision
// (compensated for float), block and grid sums in double.
template <typename T, int NW>
__global__ void __launch_bounds__(256) k_gram(VecList<T> V, VecList<T> W, size_t N, double* __restrict__ partial,
                                              unsigned int* __restrict__ counter, double* __restrict__ out) {
  __shared__ double red[32];
  constexpr int K = V16<T>::K;
  Acc<T> acc[kMaxV][NW];
  const int nv = V.nv;
  const size_t NV = N / K;          // N is a multiple of 8 (even n)
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < NV; p += (size_t)gridDim.x * blockDim.x) {
    // issue every 16-byte load of this group of K points before any use
    T w[NW][K], a[kMaxV][K];
#pragma unroll
    for (int j = 0; j < NW; ++j) ld16(W.v[j], p, w[j]);
#pragma unroll
    for (int i = 0; i < kMaxV; ++i) {
      if (i < nv) ld16(V.v[i], p, a[i]);
    }
#pragma unroll
    for (int i = 0; i < kMaxV; ++i) {
      if (i < nv) {
#pragma unroll
        for (int j = 0; j < NW; ++j)
#pragma unroll
          for (int k = 0; k < K; ++k) acc[i][j].add(a[i][k] * w[j][k]);
      }
    }
  }
  const int cols = nv * NW;
  block_sum_many<kMaxV * NW, T>(&acc[0][0], cols, partial + (size_t)blockIdx.x * cols);
  if (arrive_last(counter)) {
    block_sum_columns(partial, gridDim.x, cols, out, red);
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// out = sum_i c_i V_i; the last block writes res[0..2] = <out,out>, <out,A>, <out,B>
template <typename T>
__global__ void __launch_bounds__(256) k_lincomb(VecList<T> V, T* __restrict__ out, const T* __restrict__ A,
                                                 const T* __restrict__ B, size_t N, double* __restrict__ partial,
                                                 unsigned int* __restrict__ counter, double* __restrict__ res) {
  __shared__ double red[3 * 32];
  Acc<T> acc[3];
  const int nv = V.nv;
  T c[kMaxLin];
#pragma unroll
  for (int i = 0; i < kMaxLin; ++i) c[i] = i < nv ? (T)V.c[i] : (T)0;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
    T x[kMaxLin];
#pragma unroll
    for (int i = 0; i < kMaxLin; ++i) x[i] = i < nv ? V.v[i][p] : (T)0;
    const T av = A[p], bv = B[p];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kMaxLin; ++i) s = fma(c[i], x[i], s);
    out[p] = s;
    acc[0].add(s * s);
    acc[1].add(s * av);
    acc[2].add(s * bv);
  }
  double r[3];
  block_sum_acc<3>(acc, red, r);
  if (threadIdx.x == 0) {
    partial[(size_t)blockIdx.x * 3 + 0] = r[0];
    partial[(size_t)blockIdx.x * 3 + 1] = r[1];
    partial[(size_t)blockIdx.x * 3 + 2] = r[2];
  }
  if (arrive_last(counter)) {
    block_sum_columns(partial, gridDim.x, 3, res, red);
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// Accept a line-search step tt along d:
//   psi_t = psi + t d; g_t = 2 scale_t (gp - mu_t psi_t);
//   s = psi_t - psi (= t d); y = g_t - g; psi <- psi_t; g <- g_t;
// and, on the way, the dot products of the new pair with itself, the new
// gradient and the new psi; the last block writes res[0..5] =
//   <s,y>, <y,y>, <psi,psi>, <g,g>, <s,g>, <y,g>   (new psi, new g).
template <typename T>
__global__ void __launch_bounds__(256) k_accept(T* __restrict__ psi, const T* __restrict__ d, T tt,
                                                const T* __restrict__ gp, T a, T m,
                                                T* __restrict__ g, T* __restrict__ s, T* __restrict__ y, size_t N,
                                                double* __restrict__ partial, unsigned int* __restrict__ counter,
                                                double* __restrict__ res) {
  __shared__ double red[6 * 32];
  // tt = step, a = 2 scale_t, m = mu_t - mu_ref (converted on the host)
  constexpr int K = V16<T>::K;
  Acc<T> acc[6];
  const size_t NV = N / K;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < NV; i += (size_t)gridDim.x * blockDim.x) {
    T p0[K], dd[K], gpi[K], g0[K], pt[K], gt[K], si[K], yi[K];
    ld16(psi, i, p0); ld16(d, i, dd); ld16(gp, i, gpi); ld16(g, i, g0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      pt[k] = p0[k] + tt * dd[k];
      gt[k] = a * (gpi[k] - m * pt[k]);
      si[k] = pt[k] - p0[k];
      yi[k] = gt[k] - g0[k];
      acc[0].add(si[k] * yi[k]); acc[1].add(yi[k] * yi[k]); acc[2].add(pt[k] * pt[k]);
      acc[3].add(gt[k] * gt[k]); acc[4].add(si[k] * gt[k]); acc[5].add(yi[k] * gt[k]);
    }
    st16(s, i, si); st16(y, i, yi); st16(psi, i, pt); st16(g, i, gt);
  }
  double r[6];
  block_sum_acc<6>(acc, red, r);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 6; ++q) partial[(size_t)blockIdx.x * 6 + q] = r[q];
  }
  if (arrive_last(counter)) {
    block_sum_columns(partial, gridDim.x, 6, res, red);
    if (threadIdx.x == 0) *counter = 0u;
  }
}

}  // namespace ofdft
