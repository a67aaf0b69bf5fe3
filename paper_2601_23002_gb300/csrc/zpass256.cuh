// The z passes of the 256^3 grid (FP32 plans on the tiled path) with the
// half-length transforms held in registers.
//
// A row's real-to-complex transform along z is a complex transform of half
// length H = 128 (the even/odd packing of the generic k_zfwd / k_zinv_epi),
// here split as 128 = 16 x 8 and carried out by a team of 8 threads: each
// thread holds 16 elements (stride 8) and applies a radix-16 butterfly in
// registers, the team exchanges through a small shared-memory buffer (one pad
// element per 16 against bank conflicts; the 8 threads sit in one warp, so a
// warp barrier orders the exchange), and each thread finishes two radix-8
// butterflies with the twiddles exp(-+2 pi i j r / 128).  A 256-thread block
// runs 32 teams, one row transform each, so every thread works in every
// stage; the generic shared-memory passes leave most threads idle at this
// size (8-16 rows of 8-16 butterflies per stage) and re-read every element
// from shared memory in each stage.  All index arithmetic is compile-time.
//
// Same arithmetic as the generic pair (the packing, its split and the
// unnormalised inverse), so results agree with the generic path to FP32
// rounding; the parity tests run both against the oracle.
#pragma once
#include "passes.cuh"

namespace ofdft {

struct Z256 {
  static constexpr int N = 256, H = 128, NH = 129;
  static constexpr int A = 16, B = 8;                  // H = A * B
  static constexpr int TEAM = B;                       // threads per row transform
  static constexpr int TEAMS = 256 / TEAM;             // per 256-thread block
  static constexpr int XP = H + H / A;                 // exchange buffer per team (padded)
  static __host__ __device__ constexpr int xpos(int e) { return e + e / A; }
};

// Shared-memory bytes: twiddles W_N^k (k <= H) and W_H^k (k < H), the teams'
// exchange buffers; then the kernel's own row buffers.
template <typename T>
__host__ __device__ constexpr size_t z256_common_bytes() {
  return ((size_t)(Z256::NH + Z256::H) * sizeof(cplx<T>) + 15) / 16 * 16 +
         (size_t)Z256::TEAMS * Z256::XP * sizeof(cplx<T>);
}
template <typename T> __host__ __device__ constexpr size_t z256_fwd_bytes(int R) {
  return z256_common_bytes<T>() + 2 * (size_t)R * Z256::N * sizeof(T);
}
template <typename T> __host__ __device__ constexpr size_t z256_inv_bytes(int R, int nact) {
  return z256_common_bytes<T>() + (size_t)nact * R * Z256::NH * sizeof(cplx<T>) + 2 * (size_t)R * Z256::N * sizeof(T);
}

// 16-byte asynchronous copies of `bytes` (a multiple of 16, both ends 16-byte
// aligned) from global to shared memory by the whole block.
__device__ __forceinline__ void cp_async_block16(void* dst, const void* src, size_t bytes) {
  const int units = (int)(bytes >> 4);
  const float4* s = reinterpret_cast<const float4*>(src);
  float4* d = reinterpret_cast<float4*>(dst);
  for (int u = threadIdx.x; u < units; u += blockDim.x) cp_async<16>(d + u, s + u, true);
}

// Pass 2 of a team's transform: items j2 = j and j + 8 (of the 16), each a
// radix-8 butterfly over y[j2 + 16 r] with the twiddles W_H^(j2 r) (DIR < 0:
// forward; DIR > 0: conjugate); results u[it][r] = Z[j2 + 16 r].
template <typename T, int DIR>
__device__ __forceinline__ void z256_pass2(const cplx<T>* __restrict__ xb, const cplx<T>* __restrict__ twH, int j,
                                           cplx<T> (&u)[2][Z256::B]) {
  constexpr int A = Z256::A, B = Z256::B;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int j2 = j + B * it;
#pragma unroll
    for (int r = 0; r < B; ++r) u[it][r] = xb[j2 + (A + 1) * r];     // y[j2 + A r]
#pragma unroll
    for (int r = 1; r < B; ++r) {
      cplx<T> w = twH[j2 * r];
      if (DIR > 0) w.y = -w.y;
      u[it][r] = cmul(u[it][r], w);
    }
    Codelet<cplx<T>, B, DIR>::run(u[it]);
  }
}

// Forward z pass for n = 256 (prologue + real-to-complex along z), tiled
// layout.  smem: twN[NH] | twH[H] | xbuf[TEAMS][XP] | psit[R][N] | dbuf[R][N].
template <typename T>
__global__ void __launch_bounds__(256, 2) k_zfwd256(ProArgs<T> a, Spectra<T> sp, const cplx<T>* __restrict__ tw_h,
                                                   const cplx<T>* __restrict__ tw_n, int R) {
  constexpr int N = Z256::N, H = Z256::H, NH = Z256::NH, A = Z256::A, B = Z256::B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* twN = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* twH = twN + NH;
  cplx<T>* xbuf = reinterpret_cast<cplx<T>*>(smem_raw + (((size_t)(NH + H) * sizeof(cplx<T>) + 15) / 16 * 16));
  T* psit = reinterpret_cast<T*>(xbuf + (size_t)Z256::TEAMS * Z256::XP);
  T* dbuf = psit + (size_t)R * N;
  const size_t row0 = (size_t)blockIdx.x * R;        // R divides N * N
  const size_t off = row0 * N;
  const T* src0 = a.mode == 0 ? a.rho : a.psi;
  const bool has_d = a.mode != 0 && a.d != nullptr;
  cp_async_block16(psit, src0 + off, (size_t)R * N * sizeof(T));
  if (has_d) cp_async_block16(dbuf, a.d + off, (size_t)R * N * sizeof(T));
  for (int q = threadIdx.x; q < NH + H; q += blockDim.x) twN[q] = q < NH ? tw_n[q] : tw_h[q - NH];
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  const T tstep = a.dsc ? (T)a.dsc[2] : a.t;
  for (int q = threadIdx.x; q < R * N; q += blockDim.x) {
    const T x = psit[q];
    if (a.mode == 0) { dbuf[q] = x; psit[q] = sqrt(fmax(x, (T)0)); }
    else if (has_d) psit[q] = x + tstep * dbuf[q];
  }
  __syncthreads();
  const T scale = a.dsc ? (T)a.dsc[0] : a.scale, alpha = a.alpha, nmin = (T)kNmin;
  const T psi_shift = a.dsc ? (T)a.dsc[1] : a.psi_shift;
  const int team = threadIdx.x / B, j = threadIdx.x % B;
  cplx<T>* xb = xbuf + (size_t)team * Z256::XP;
  const int ntr = R * sp.nact;
  for (int t0 = 0; t0 < ntr; t0 += Z256::TEAMS) {
    const int t = t0 + team;
    const bool act = t < ntr;                          // the whole team alike
    const int f = act ? t / R : 0, r = act ? t - f * R : 0;
    const int fid = sp.idx[f];
    cplx<T> u[2][B];
    if (act) {
      // pass 1: z_m = (x_2m, x_2m+1) at m = j + 8 s, radix 16
      cplx<T> v[A];
      const T* pr = psit + r * N;
      const T* dr = dbuf + r * N;
#pragma unroll
      for (int s = 0; s < A; ++s) {
        const int m = j + B * s;
        T x0 = pr[2 * m], x1 = pr[2 * m + 1];
        if (fid == 2) {
          x0 -= psi_shift; x1 -= psi_shift;
        } else {
          T n0, n1;
          if (a.mode == 0) { n0 = dr[2 * m]; n1 = dr[2 * m + 1]; }
          else { n0 = scale * x0 * x0; n1 = scale * x1 * x1; }
          if (fid == 0) { x0 = n0; x1 = n1; }
          else { x0 = pow_t<T>(fmax(n0, nmin), alpha); x1 = pow_t<T>(fmax(n1, nmin), alpha); }
        }
        v[s] = mk<T>(x0, x1);
      }
      Codelet<cplx<T>, A, -1>::run(v);
#pragma unroll
      for (int s = 0; s < A; ++s) xb[j * (A + 1) + s] = v[s];        // y[j A + s]
    }
    __syncwarp();
    if (act) {
      z256_pass2<T, -1>(xb, twH, j, u);
      // Z[j2 + 16 r] back into the slots this thread read
#pragma unroll
      for (int it = 0; it < 2; ++it)
#pragma unroll
        for (int rr = 0; rr < B; ++rr) xb[j + B * it + (A + 1) * rr] = u[it][rr];
    }
    __syncwarp();
    if (act) {
      // X[k] = (Z[k] + Z*[H-k])/2 - (i/2) W_N^k (Z[k] - Z*[H-k]), k = 0..H (Z[H] = Z[0])
      cplx<T>* out = sp.s[fid] + (row0 + r) * NH;
#pragma unroll
      for (int s = 0; s <= A; ++s) {
        const int k = j + B * s;
        if (s == A && j != 0) break;                   // k = H: thread 0 only
        const cplx<T> zk = xb[Z256::xpos(k == H ? 0 : k)];
        const cplx<T> zc = cconj(xb[Z256::xpos(k == 0 ? 0 : H - k)]);
        const cplx<T> e = cadd(zk, zc);
        const cplx<T> wo = cmul(twN[k], csub(zk, zc));
        out[k] = mk<T>((T)0.5 * (e.x + wo.y), (T)0.5 * (e.y - wo.x));
      }
    }
    __syncwarp();                                      // xb is rewritten by the next round
  }
}

// Inverse z pass for n = 256 (complex-to-real along z) fused with the
// pointwise functional, tiled layout.
// smem: twN[NH] | twH[H] | xbuf[TEAMS][XP] | stg[nact][R][NH] | pin[2][R][N].
// A row's real output overwrites its own staging row (pitch 2 NH reals).
template <typename T>
__global__ void __launch_bounds__(256, 2) k_zinv256(Spectra<T> sp, EpiArgs<T> a, const cplx<T>* __restrict__ tw_h,
                                                   const cplx<T>* __restrict__ tw_n, int R) {
  constexpr int N = Z256::N, H = Z256::H, NH = Z256::NH, A = Z256::A, B = Z256::B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* twN = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* twH = twN + NH;
  cplx<T>* xbuf = reinterpret_cast<cplx<T>*>(smem_raw + (((size_t)(NH + H) * sizeof(cplx<T>) + 15) / 16 * 16));
  cplx<T>* stg = xbuf + (size_t)Z256::TEAMS * Z256::XP;
  T* pin = reinterpret_cast<T*>(stg + (size_t)sp.nact * R * NH);
  const size_t row0 = (size_t)blockIdx.x * R;
  const size_t off = row0 * N;
  // spectra rows (contiguous per field: R NH complex, 16-byte aligned since R is even)
  for (int f = 0; f < sp.nact; ++f)
    cp_async_block16(stg + (size_t)f * R * NH, sp.s[sp.idx[f]] + row0 * NH, (size_t)R * NH * sizeof(cplx<T>));
  {
    const T* src0 = a.mode == 0 ? a.rho : (a.mode == 3 ? a.pold : a.psi);
    if (a.mode != 3 || a.pyout) cp_async_block16(pin, src0 + off, (size_t)R * N * sizeof(T));
    if (a.mode == 1) cp_async_block16(pin + (size_t)R * N, a.d + off, (size_t)R * N * sizeof(T));
  }
  for (int q = threadIdx.x; q < NH + H; q += blockDim.x) twN[q] = q < NH ? tw_n[q] : tw_h[q - NH];
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  const int team = threadIdx.x / B, j = threadIdx.x % B;
  cplx<T>* xb = xbuf + (size_t)team * Z256::XP;
  const int ntr = R * sp.nact;
  for (int t0 = 0; t0 < ntr; t0 += Z256::TEAMS) {
    const int t = t0 + team;
    const bool act = t < ntr;
    const int f = act ? t / R : 0, r = act ? t - f * R : 0;
    cplx<T>* in = stg + ((size_t)f * R + r) * NH;
    if (act) {
      // Z[k] = (X[k] + X*[H-k]) + i W_N^-k (X[k] - X*[H-k]) at k = j + 8 s, radix 16
      cplx<T> v[A];
#pragma unroll
      for (int s = 0; s < A; ++s) {
        const int k = j + B * s;
        const cplx<T> xk = in[k];
        const cplx<T> xc = cconj(in[H - k]);
        const cplx<T> e = cadd(xk, xc);
        const cplx<T> o = cmul(cconj(twN[k]), csub(xk, xc));
        v[s] = mk<T>(e.x - o.y, e.y + o.x);
      }
      Codelet<cplx<T>, A, +1>::run(v);
#pragma unroll
      for (int s = 0; s < A; ++s) xb[j * (A + 1) + s] = v[s];
    }
    __syncwarp();                                      // (the team has read its staging row)
    if (act) {
      cplx<T> u[2][B];
      z256_pass2<T, +1>(xb, twH, j, u);
      // z[m], m = j2 + 16 r: the real pair (x_2m, x_2m+1) into the staging row
#pragma unroll
      for (int it = 0; it < 2; ++it)
#pragma unroll
        for (int rr = 0; rr < B; ++rr) in[j + B * it + A * rr] = u[it][rr];
    }
    __syncwarp();
  }
  __syncthreads();
  const int rp = 2 * NH;                               // real row pitch in the staging slots
  T* realf[3] = {nullptr, nullptr, nullptr};
  for (int f = 0; f < sp.nact; ++f) realf[sp.idx[f]] = reinterpret_cast<T*>(stg + (size_t)f * R * NH);
  const int jt = threadIdx.x;                          // one grid point of each row (blockDim = N)
  if (a.mode == 3) {
    const T* fP = realf[2];
    for (int r = 0; r < R; ++r) {
      const T v = fP[r * rp + jt];
      a.out[off + r * N + jt] = v;
      if (a.pyout) a.pyout[off + r * N + jt] = v - pin[r * N + jt];
    }
    return;
  }
  const EpiPoint<T> ep(sp, a);
  AccShort<T> acc[8];
  const T* pd = pin + (size_t)R * N;
  for (int r = 0; r < R; ++r) {
    const int qs = r * rp + jt, q = r * N + jt;
    ep.point(a, pin[q], a.mode != 0 ? pd[q] : (T)0, realf[0] ? realf[0][qs] : (T)0,
             realf[1] ? realf[1][qs] : (T)0, realf[2] ? realf[2][qs] : (T)0, off + q, acc);
  }
  typename TreeVal<T>::type* scr = reinterpret_cast<typename TreeVal<T>::type*>(smem_raw);
  block_sum_tree_raw<8, T>(acc, a.partials + (size_t)blockIdx.x * 8, scr);
  if (arrive_last(a.counter)) {
    finalize_eval<T>(a.fin, scr);
    if (threadIdx.x == 0) *a.counter = 0u;
  }
}

}  // namespace ofdft
