// Grid-vector kernels of the minimiser: fused multi-dot products, linear
// combinations and the L-BFGS accept step.  FP64 accumulation throughout.
#pragma once
#include "common.cuh"

namespace ofdft {

constexpr int kMaxV = 9;    // vectors per gram launch (longer lists are chunked)
constexpr int kMaxW = 4;    // targets per gram launch
constexpr int kMaxLin = 40; // terms of a linear combination

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

// All dot products <V_i, W_j>, i < nv <= kMaxV, j < NW.  partial[block][i*NW + j].
template <typename T, int NW>
__global__ void __launch_bounds__(256) k_gram(VecList<T> V, VecList<T> W, size_t N, double* __restrict__ partial) {
  __shared__ double red[32];
  double acc[kMaxV][NW];
#pragma unroll
  for (int i = 0; i < kMaxV; ++i)
#pragma unroll
    for (int j = 0; j < NW; ++j) acc[i][j] = 0;
  const int nv = V.nv;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
    double w[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) w[j] = (double)W.v[j][p];
#pragma unroll
    for (int i = 0; i < kMaxV; ++i) {
      if (i < nv) {
        const double a = (double)V.v[i][p];
#pragma unroll
        for (int j = 0; j < NW; ++j) acc[i][j] = fma(a, w[j], acc[i][j]);
      }
    }
  }
  // block reduction one value at a time (warp shuffles, then lane 0 of each warp)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < kMaxV; ++i) {
    if (i >= nv) break;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      double s = warp_sum(acc[i][j]);
      __syncthreads();
      if (lane == 0) red[wid] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0;
        for (int k = 0; k < nwarp; ++k) t += red[k];
        partial[(size_t)blockIdx.x * (nv * NW) + i * NW + j] = t;
      }
    }
  }
}

// out = sum_i c_i V_i; partial[block][0..2] = <out,out>, <out,A>, <out,B>
template <typename T>
__global__ void __launch_bounds__(256) k_lincomb(VecList<T> V, T* __restrict__ out, const T* __restrict__ A,
                                                 const T* __restrict__ B, size_t N, double* __restrict__ partial) {
  __shared__ double red[3 * 32];
  double acc[3] = {0, 0, 0};
  const int nv = V.nv;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int i = 0; i < nv; ++i) s = fma(V.c[i], (double)V.v[i][p], s);
    const T o = (T)s;
    out[p] = o;
    const double od = (double)o;
    acc[0] = fma(od, od, acc[0]);
    acc[1] = fma(od, (double)A[p], acc[1]);
    acc[2] = fma(od, (double)B[p], acc[2]);
  }
  double r[3];
  block_sum<3>(acc, red, r);
  if (threadIdx.x == 0) {
    partial[(size_t)blockIdx.x * 3 + 0] = r[0];
    partial[(size_t)blockIdx.x * 3 + 1] = r[1];
    partial[(size_t)blockIdx.x * 3 + 2] = r[2];
  }
}

// Accept a line-search step t along d:
//   psi_t = psi + t d; g_t = 2 scale_t (gp - mu_t psi_t);
//   s = psi_t - psi (= t d); y = g_t - g; psi <- psi_t; g <- g_t.
template <typename T>
__global__ void k_accept(T* __restrict__ psi, const T* __restrict__ d, double t, const T* __restrict__ gp,
                         double scale_t, double mu_t, T* __restrict__ g, T* __restrict__ s, T* __restrict__ y,
                         size_t N) {
  const T tt = (T)t, a = (T)(2.0 * scale_t), m = (T)mu_t;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const T p0 = psi[i];
    const T pt = p0 + tt * d[i];
    const T gt = a * (gp[i] - m * pt);
    if (s) s[i] = pt - p0;
    if (y) y[i] = gt - g[i];
    psi[i] = pt;
    g[i] = gt;
  }
}

}  // namespace ofdft
