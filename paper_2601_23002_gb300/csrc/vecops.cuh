// Grid-vector kernels of the minimiser: fused multi-dot products, linear
// combinations and the L-BFGS accept step.  FP64 accumulation throughout.
#pragma once
#include "common.cuh"

namespace ofdft {

constexpr int kMaxV = 16;   // vectors per gram launch (longer lists are chunked)
constexpr int kMaxW = 5;    // targets per gram launch
constexpr int kMaxLin = 20; // vectors of one streamed list: a combination's 1 + 2 m <= 17 terms and its
                            // two dot targets, or kMaxV Gram vectors and kMaxW targets

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

// The three streaming passes below read their vectors through a per-thread
// ring of asynchronous copies (cp.async, 16 bytes per vector per thread) in
// shared memory: S-1 groups' copies are in flight while the thread works on
// the current one, without holding them in registers, so one 256-thread block
// per SM keeps 70-140 KB in flight with ~100 registers per thread.  Each
// thread reads back only what it copied itself, so the ring needs no block
// barrier.  Ring layout: [S][nvec][blockDim] groups of 16 bytes.
constexpr int kStreamThreads = 256;
template <typename T> struct StreamCfg {
  using V = typename V16<T>::type;                 // one 16-byte group (4 floats or 2 doubles)
  static constexpr int K = V16<T>::K;
  static constexpr size_t ring_bytes(int S, int nvec) { return (size_t)S * nvec * kStreamThreads * 16; }
};
// stages for a list of nvec vectors: as many as ~200 KB of ring allows
__host__ __device__ constexpr int stream_stages(int nvec) { return nvec <= 4 ? 8 : nvec <= 17 ? 3 : 2; }

template <typename T>
__device__ __forceinline__ void lds16(const typename V16<T>::type* p, T (&o)[V16<T>::K]) {
  const typename V16<T>::type v = *p;
  memcpy(o, &v, sizeof(o));
}

// Groups p = blockIdx.x * blockDim.x + threadIdx.x + k * (gridDim.x *
// blockDim.x) of the nvec <= kMaxLin vectors src.v[] (N elements each,
// 16-byte aligned, N a multiple of the group size).  For every group the
// thread calls body(mine, p), where mine[i * blockDim.x] is vector i's group
// p in shared memory.
template <typename T, int S, typename List, typename Body>
__device__ __forceinline__ void cpa_stream(const List& src, int nvec, size_t N, unsigned char* smem, Body&& body) {
  using V = typename V16<T>::type;
  constexpr int K = V16<T>::K;
  V* buf = reinterpret_cast<V*>(smem);
  const size_t NG = N / K;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t p0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t iters = p0 < NG ? (NG - p0 + stride - 1) / stride : 0;
  const size_t stage = (size_t)nvec * blockDim.x;
  auto issue = [&](size_t k) {
    V* dst = buf + (size_t)(k % S) * stage + threadIdx.x;
    const size_t p = p0 + k * stride;
#pragma unroll
    for (int i = 0; i < kMaxLin; ++i)
      if (i < nvec) cp_async<16>(dst + (size_t)i * blockDim.x, reinterpret_cast<const V*>(src.v[i]) + p, true);
  };
#pragma unroll
  for (int k = 0; k < S - 1; ++k) {
    if ((size_t)k < iters) issue(k);
    cp_async_commit();
  }
  for (size_t k = 0; k < iters; ++k) {
    // the slot refilled here was last read by this thread in iteration k-1
    if (k + S - 1 < iters) issue(k + S - 1);
    cp_async_commit();
    cp_async_wait<S - 1>();
    body(buf + (size_t)(k % S) * stage + threadIdx.x, p0 + k * stride);
  }
  cp_async_wait<0>();
}

// All dot products <X_i, X_{nv+j}>, i < nv <= kMaxV, j < NW (X lists the nv
// vectors, then the NW targets).  Per block into partial[block][i*NW + j]; the
// last block sums the columns into out[] in a fixed order.  The products of a
// group's K elements are summed in the vectors' precision and added to a
// compensated per-thread sum (float); block and grid sums in double.
template <typename T, int NW, int S>
__global__ void __launch_bounds__(kStreamThreads, 1)
k_gram(VecList<T> X, int nv, size_t N, double* __restrict__ partial, unsigned int* __restrict__ counter,
       double* __restrict__ out) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[32];
  using V = typename V16<T>::type;
  constexpr int K = V16<T>::K;
  Acc<T> acc[kMaxV][NW];
  cpa_stream<T, S>(X, nv + NW, N, smem, [&](const V* mine, size_t) {
    T w[NW][K];
#pragma unroll
    for (int j = 0; j < NW; ++j) lds16<T>(mine + (size_t)(nv + j) * kStreamThreads, w[j]);
#pragma unroll
    for (int i = 0; i < kMaxV; ++i) {
      if (i < nv) {
        T a[K];
        lds16<T>(mine + (size_t)i * kStreamThreads, a);
#pragma unroll
        for (int j = 0; j < NW; ++j) {
          T t = a[0] * w[j][0];
#pragma unroll
          for (int k = 1; k < K; ++k) t = fma(a[k], w[j][k], t);
          acc[i][j].add(t);
        }
      }
    }
  });
  const int cols = nv * NW;
  // the ring is free: reuse it as reduction scratch (the host checks its size)
  block_sum_tree<kMaxV * NW, T>(&acc[0][0], cols, partial + (size_t)blockIdx.x * cols,
                                reinterpret_cast<typename TreeVal<T>::type*>(smem));
  if (arrive_last(counter)) {
    block_sum_columns(partial, gridDim.x, cols, out, red);
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// The scale of a line-search trial psi + t d (n = N_e (psi + t d)^2 / Q(t),
// Q(t) = Q + 2 t <d,psi> + t^2 <d,d>) and the mean-psi shift sqrt(nbar/scale),
// formed on the device from the direction's dots so that the first trial can
// be launched without a host round trip.  out == nullptr: not wanted.
struct TrialScale {
  double q, t, ne, dv, nbar;
  double* out;       // out[0] = scale, out[1] = sqrt(nbar / scale), out[2] = t
  // when set: q = *qdev, and t = 1 if *kkdev > 0 (a quasi-Newton step), else
  // the first step 0.1 sqrt(q / <d,d>) (10% of |psi| along -P g)
  const double* qdev;
  const int* kkdev;
};

// L-BFGS history scalars kept on the device, indexed by ring slot (< 8):
// <s_a, y_b>, <y_a, y_b>, <y_a, P y_b>, and <s, g>, <y, g>, <y, P g> for the
// current g; Q = int psi^2; the recursion's gamma, pairs used (kk) and the
// direction's coefficients (P g first, then (P y_j, s_j) in ring order).
constexpr int kTLMax = 8;
struct TwoLoopState {
  double SY[kTLMax * kTLMax], YY[kTLMax * kTLMax], YPY[kTLMax * kTLMax];
  double Sg[kTLMax], Yg[kTLMax], YPg[kTLMax];
  double Q, gamma;
  double coef[1 + 2 * kTLMax];
  int kk;
};
struct TwoLoopArgs {
  int count;                  // pairs in the ring, the new one included
  int new_slot;               // slot of the pair accepted last
  int no;                     // older pairs
  int old_slot[kTLMax];       // their slots, ring order
  int ring_slot[kTLMax];      // all slots, ring order (oldest first)
  double dv;
};

// One warp, FP64: fold the new pair into the history scalars from
// acc[0..5] = k_accept's <s,y>, <y,y>, Q, <g,g>, <s,g>, <y,g> and the Gram
// pass's cross[row * 4 + col], rows [older s, older y, y_new], columns
// [g, P g, y_new, P y_new] (raw sums, times dv here).  The recursion reads
// <s_a, y_b> only for a older than b, <y, y> only on the newest pair, and
// <y, P y>, <y, P g>, <s, g>; nothing else is kept.  Then the two-loop
// recursion with H0 = gamma P on those scalars:
//   q = g - sum alpha_j y_j,  d = -(gamma P q + sum (alpha_j - beta_j) s_j),
//   P q = P g - sum alpha_k P y_k,  <y_i, P q> = <y_i, P g> - sum alpha_k <y_i, P y_k>.
// A new pair without positive curvature drops the history (kk = 0, d = -P g).
// The state is staged in shared memory by the whole warp, and the recursion
// runs with one lane per pair.  res[0] = gamma, res[1] = kk.
static __global__ void __launch_bounds__(32) k_twoloop(TwoLoopArgs a, const double* __restrict__ cross,
                                                       const double* __restrict__ acc,
                                                       TwoLoopState* __restrict__ st, double* __restrict__ res) {
  constexpr int M2 = kTLMax * kTLMax;
  __shared__ double sSY[M2], sYY[M2], sYPY[M2], sSg[kTLMax], sYg[kTLMax], sYPg[kTLMax];
  __shared__ double sX[(2 * kTLMax + 1) * 4], sA[6], srho[kTLMax], scoef[1 + 2 * kTLMax];
  __shared__ double sgam;
  __shared__ int skk;
  const int lane = threadIdx.x;
  const int no = a.no, ns = a.new_slot;
  const double dv = a.dv;
  for (int q = lane; q < M2; q += 32) { sSY[q] = st->SY[q]; sYY[q] = st->YY[q]; sYPY[q] = st->YPY[q]; }
  if (lane < kTLMax) { sSg[lane] = st->Sg[lane]; sYg[lane] = st->Yg[lane]; sYPg[lane] = st->YPg[lane]; }
  for (int q = lane; q < (2 * no + 1) * 4; q += 32) sX[q] = cross[q] * dv;
  if (lane < 6) sA[lane] = acc[lane] * dv;
  __syncwarp();
  // the new pair's rows and columns (lane i < no: older pair i; lane 31: own dots)
  if (lane < no) {
    const int si = a.old_slot[lane];
    const int i = lane;
    sSg[si] = sX[i * 4 + 0];                                   // <s_i, g>
    sSY[si * kTLMax + ns] = sX[i * 4 + 2];                     // <s_i, y_new>
    sYg[si] = sX[(no + i) * 4 + 0];                            // <y_i, g>
    sYPg[si] = sX[(no + i) * 4 + 1];                           // <y_i, P g>
    sYPY[si * kTLMax + ns] = sYPY[ns * kTLMax + si] = sX[(no + i) * 4 + 3];   // <y_i, P y_new>
  } else if (lane == 31) {
    sSY[ns * kTLMax + ns] = sA[0];
    sYY[ns * kTLMax + ns] = sA[1];
    sSg[ns] = sA[4];
    sYg[ns] = sA[5];
    sYPg[ns] = sX[2 * no * 4 + 1];
    sYPY[ns * kTLMax + ns] = sX[2 * no * 4 + 3];
  }
  __syncwarp();
  const int kk = sSY[ns * kTLMax + ns] > 0 ? a.count : 0;
  // reciprocals of the curvatures, one lane each
  if (lane < kk) { const int sl = a.ring_slot[lane]; srho[lane] = 1.0 / sSY[sl * kTLMax + sl]; }
  if (lane == 8 && kk > 0) {
    const int sl = a.ring_slot[kk - 1];
    sgam = sSY[sl * kTLMax + sl] / sYY[sl * kTLMax + sl];
  }
  __syncwarp();
  // the recursion with lane i holding pair i (ring order): each alpha_j (and
  // later alpha_j - beta_j) is broadcast as soon as it is final and the other
  // lanes fold it in, so the dependent chain is ~2 kk steps long
  const unsigned FULL = 0xffffffffu;
  const bool mine = lane < kk;
  const int rl = mine ? a.ring_slot[lane] : 0;
  const double gamma = kk > 0 ? sgam : 1.0;
  double sq = mine ? sSg[rl] : 0.0, alpha_l = 0.0;
  for (int j = kk - 1; j >= 0; --j) {
    if (lane == j) alpha_l = srho[j] * sq;
    const double aj = __shfl_sync(FULL, alpha_l, j);
    if (lane < j) sq -= aj * sSY[rl * kTLMax + a.ring_slot[j]];
  }
  // <y_l, P q> = <y_l, P g> - sum_k alpha_k <y_l, P y_k>, independent per lane
  double ypq = mine ? sYPg[rl] : 0.0;
  for (int k = 0; k < kk; ++k) {
    const double ak = __shfl_sync(FULL, alpha_l, k);
    if (mine) ypq -= ak * sYPY[rl * kTLMax + a.ring_slot[k]];
  }
  double yr = gamma * ypq, beta_l = 0.0;
  for (int i = 0; i < kk; ++i) {
    if (lane == i) beta_l = srho[i] * yr;
    const double di = __shfl_sync(FULL, alpha_l - beta_l, i);
    if (lane > i && mine) yr += di * sSY[a.ring_slot[i] * kTLMax + rl];
  }
  if (lane == 0) scoef[0] = kk > 0 ? -gamma : -1.0;
  if (lane < kTLMax) {
    scoef[1 + 2 * lane] = mine ? gamma * alpha_l : 0.0;
    scoef[2 + 2 * lane] = mine ? -(alpha_l - beta_l) : 0.0;
  }
  if (lane == 0) { sgam = gamma; skk = kk; }
  __syncwarp();
  for (int q = lane; q < M2; q += 32) { st->SY[q] = sSY[q]; st->YY[q] = sYY[q]; st->YPY[q] = sYPY[q]; }
  if (lane < kTLMax) { st->Sg[lane] = sSg[lane]; st->Yg[lane] = sYg[lane]; st->YPg[lane] = sYPg[lane]; }
  if (lane < 1 + 2 * kTLMax) st->coef[lane] = scoef[lane];
  if (lane == 0) {
    st->Q = sA[2];
    st->gamma = sgam;
    st->kk = skk;
    res[0] = sgam;
    res[1] = (double)skk;
  }
}

// out = sum_{i < nv} c_i X_i, with X_nv = A and X_{nv+1} = B; the last block
// writes res[0..2] = <out,out>, <out,A>, <out,B> (raw sums, without dV) and,
// with B = psi, the trial scale of ts
template <typename T>
__global__ void __launch_bounds__(kStreamThreads, 1)
k_lincomb(VecList<T> X, int nv, T* __restrict__ out, size_t N, double* __restrict__ partial,
          unsigned int* __restrict__ counter, double* __restrict__ res, TrialScale ts,
          const double* __restrict__ dcoef) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[32];
  using V = typename V16<T>::type;
  constexpr int K = V16<T>::K;
  Acc<T> acc[3];
  T c[kMaxLin - 2];
#pragma unroll
  for (int i = 0; i < kMaxLin - 2; ++i) c[i] = i < nv ? (T)(dcoef ? dcoef[i] : X.c[i]) : (T)0;
  cpa_stream<T, stream_stages(kMaxLin - 1)>(X, nv + 2, N, smem, [&](const V* mine, size_t p) {
    T s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = 0;
#pragma unroll
    for (int i = 0; i < kMaxLin - 2; ++i) {
      if (i < nv) {
        T x[K];
        lds16<T>(mine + (size_t)i * kStreamThreads, x);
#pragma unroll
        for (int k = 0; k < K; ++k) s[k] = fma(c[i], x[k], s[k]);
      }
    }
    T av[K], bv[K];
    lds16<T>(mine + (size_t)nv * kStreamThreads, av);
    lds16<T>(mine + (size_t)(nv + 1) * kStreamThreads, bv);
    st16(out, p, s);
    T t0 = s[0] * s[0], t1 = s[0] * av[0], t2 = s[0] * bv[0];
#pragma unroll
    for (int k = 1; k < K; ++k) {
      t0 = fma(s[k], s[k], t0); t1 = fma(s[k], av[k], t1); t2 = fma(s[k], bv[k], t2);
    }
    acc[0].add(t0); acc[1].add(t1); acc[2].add(t2);
  });
  block_sum_tree<3, T>(acc, 3, partial + (size_t)blockIdx.x * 3, reinterpret_cast<typename TreeVal<T>::type*>(smem));
  if (arrive_last(counter)) {
    block_sum_columns(partial, gridDim.x, 3, res, red);
    if (threadIdx.x == 0) *counter = 0u;
    if (ts.out) {
      __syncthreads();                   // res[] written by this block's threads
      if (threadIdx.x == 0) {
        const double dd = res[0] * ts.dv, dpsi = res[2] * ts.dv;
        const double q = ts.qdev ? *ts.qdev : ts.q;
        double t = ts.t;
        if (ts.kkdev && *ts.kkdev == 0) t = 0.1 * sqrt(q / fmax(dd, 1e-300));
        const double sc = ts.ne / (q + 2.0 * t * dpsi + t * t * dd);
        ts.out[0] = sc;
        ts.out[1] = sqrt(ts.nbar / sc);
        ts.out[2] = t;
      }
    }
  }
}

// Accept a line-search step tt along d (X = {psi, d, gp, g}):
//   psi_t = psi + t d; g_t = 2 scale_t (gp - mu_t psi_t);
//   s = psi_t - psi (= t d); y = g_t - g; psi <- psi_t; g <- g_t;
// and, on the way, the dot products of the new pair with itself, the new
// gradient and the new psi; the last block writes res[0..5] =
//   <s,y>, <y,y>, <psi,psi>, <g,g>, <s,g>, <y,g>   (new psi, new g).
// A thread rewrites psi and g only at the groups it has already copied in.
template <typename T>
__global__ void __launch_bounds__(kStreamThreads, 1)
k_accept(VecList<T> X, T tt, T a, T m, T* __restrict__ psi, T* __restrict__ g, T* __restrict__ s,
         T* __restrict__ y, size_t N, double* __restrict__ partial, unsigned int* __restrict__ counter,
         double* __restrict__ res) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[32];
  // tt = step, a = 2 scale_t, m = mu_t - mu_ref (converted on the host)
  using V = typename V16<T>::type;
  constexpr int K = V16<T>::K;
  Acc<T> acc[6];
  cpa_stream<T, stream_stages(4)>(X, 4, N, smem, [&](const V* mine, size_t p) {
    T p0[K], dd[K], gpi[K], g0[K], pt[K], gt[K], si[K], yi[K];
    lds16<T>(mine, p0);
    lds16<T>(mine + kStreamThreads, dd);
    lds16<T>(mine + 2 * kStreamThreads, gpi);
    lds16<T>(mine + 3 * kStreamThreads, g0);
    T t[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < K; ++k) {
      pt[k] = p0[k] + tt * dd[k];
      gt[k] = a * (gpi[k] - m * pt[k]);
      si[k] = pt[k] - p0[k];
      yi[k] = gt[k] - g0[k];
      t[0] = fma(si[k], yi[k], t[0]); t[1] = fma(yi[k], yi[k], t[1]); t[2] = fma(pt[k], pt[k], t[2]);
      t[3] = fma(gt[k], gt[k], t[3]); t[4] = fma(si[k], gt[k], t[4]); t[5] = fma(yi[k], gt[k], t[5]);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[q].add(t[q]);
    st16(s, p, si); st16(y, p, yi); st16(psi, p, pt); st16(g, p, gt);
  });
  block_sum_tree<6, T>(acc, 6, partial + (size_t)blockIdx.x * 6, reinterpret_cast<typename TreeVal<T>::type*>(smem));
  if (arrive_last(counter)) {
    block_sum_columns(partial, gridDim.x, 6, res, red);
    if (threadIdx.x == 0) *counter = 0u;
  }
}

}  // namespace ofdft
