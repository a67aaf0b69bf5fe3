// The passes of the 256^3 grid (FP32 plans) with their transforms held in
// registers: the z passes below; then the x-y transforms with the G-space
// terms, either on one kz plane per cluster of eight blocks (plane layout,
// k_plane256cl, the default) or as the y pass and the x pass on tiles (tiled
// layout, k_ypass256 / k_xgspace256).
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
#include <cooperative_groups.h>
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
template <typename T> __host__ __device__ constexpr size_t z256_fwd_bytes(int /*R: no row buffers*/) {
  return z256_common_bytes<T>();
}
template <typename T> __host__ __device__ constexpr size_t z256_inv_bytes(int R, int nact) {
  return z256_common_bytes<T>() + (size_t)nact * R * Z256::NH * sizeof(cplx<T>);
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

// Forward z pass for n = 256 (prologue + real-to-complex along z), tiled or
// plane layout (Spectra::planes); R rows per block (8, 16 or 32: a template
// parameter, so the row arithmetic is shifts and masks).  Each team reads its
// row's pairs (x_2m, x_2m+1) straight from memory (rho, or psi and d) and
// forms the field's input in registers.  smem: twN[NH] | twH[H] | xbuf[TEAMS][XP]
// (37 KB: four blocks per SM).
template <typename T, int R>
__global__ void __launch_bounds__(256, 4) k_zfwd256(ProArgs<T> a, Spectra<T> sp, const cplx<T>* __restrict__ tw_h,
                                                   const cplx<T>* __restrict__ tw_n) {
  constexpr int N = Z256::N, H = Z256::H, NH = Z256::NH, A = Z256::A, B = Z256::B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* twN = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* twH = twN + NH;
  cplx<T>* xbuf = reinterpret_cast<cplx<T>*>(smem_raw + (((size_t)(NH + H) * sizeof(cplx<T>) + 15) / 16 * 16));
  const size_t row0 = (size_t)blockIdx.x * R;        // R divides N * N
  const size_t off = row0 * N;
  const T* src0 = a.mode == 0 ? a.rho : a.psi;
  const bool has_d = a.mode != 0 && a.d != nullptr;
  for (int q = threadIdx.x; q < NH + H; q += blockDim.x) twN[q] = q < NH ? tw_n[q] : tw_h[q - NH];
  __syncthreads();
  const T tstep = a.dsc ? (T)a.dsc[2] : a.t;
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
      const float2* pr = reinterpret_cast<const float2*>(src0 + off + (size_t)r * N);
      const float2* dr = has_d ? reinterpret_cast<const float2*>(a.d + off + (size_t)r * N) : nullptr;
      float2 w[A];
#pragma unroll
      for (int s = 0; s < A; ++s) w[s] = __ldg(pr + j + B * s);
      if (has_d) {
#pragma unroll
        for (int s = 0; s < A; ++s) {
          const float2 dd = __ldg(dr + j + B * s);
          w[s].x = w[s].x + tstep * dd.x; w[s].y = w[s].y + tstep * dd.y;
        }
      }
#pragma unroll
      for (int s = 0; s < A; ++s) {
        T x0 = w[s].x, x1 = w[s].y;
        if (fid == 2) {
          if (a.mode == 0) { x0 = sqrt(fmax(x0, (T)0)); x1 = sqrt(fmax(x1, (T)0)); }
          x0 -= psi_shift; x1 -= psi_shift;
        } else {
          T n0, n1;
          if (a.mode == 0) { n0 = x0; n1 = x1; }
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
      // X[k] = (Z[k] + Z*[H-k])/2 - (i/2) W_N^k (Z[k] - Z*[H-k]), k = 0..H (Z[H] = Z[0]);
      // plane layout: entry (k, row) at k N^2 + row (the four teams of a
      // warp, consecutive rows, fill whole 32-byte sectors)
      cplx<T>* out = sp.planes ? sp.s[fid] + row0 + r : sp.s[fid] + (row0 + r) * NH;
      const size_t kstride = sp.planes ? (size_t)N * N : 1;
#pragma unroll
      for (int s = 0; s <= A; ++s) {
        const int k = j + B * s;
        if (s == A && j != 0) break;                   // k = H: thread 0 only
        const cplx<T> zk = xb[Z256::xpos(k == H ? 0 : k)];
        const cplx<T> zc = cconj(xb[Z256::xpos(k == 0 ? 0 : H - k)]);
        const cplx<T> e = cadd(zk, zc);
        const cplx<T> wo = cmul(twN[k], csub(zk, zc));
        out[k * kstride] = mk<T>((T)0.5 * (e.x + wo.y), (T)0.5 * (e.y - wo.x));
      }
    }
    __syncwarp();                                      // xb is rewritten by the next round
  }
}

// Inverse z pass for n = 256 (complex-to-real along z) fused with the
// pointwise functional, tiled or plane layout.
// smem: twN[NH] | twH[H] | xbuf[TEAMS][XP] | stg[nact][R][NH].
// A row's real output overwrites its own staging row (pitch 2 NH reals).
// The real-space inputs (rho, or psi and d; P g's previous value) are read
// straight from memory in the pointwise loop, one row ahead, rather than
// staged: 33 KB less shared memory per block at 16 rows, three blocks per SM
// instead of two.
template <typename T, int R>
__global__ void __launch_bounds__(256, 3) k_zinv256(Spectra<T> sp, EpiArgs<T> a, const cplx<T>* __restrict__ tw_h,
                                                   const cplx<T>* __restrict__ tw_n) {
  constexpr int N = Z256::N, H = Z256::H, NH = Z256::NH, A = Z256::A, B = Z256::B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* twN = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* twH = twN + NH;
  cplx<T>* xbuf = reinterpret_cast<cplx<T>*>(smem_raw + (((size_t)(NH + H) * sizeof(cplx<T>) + 15) / 16 * 16));
  cplx<T>* stg = xbuf + (size_t)Z256::TEAMS * Z256::XP;
  const size_t row0 = (size_t)blockIdx.x * R;
  const size_t off = row0 * N;
  // spectra rows: tiled layout, contiguous per field (R NH complex, 16-byte
  // aligned since R is even); plane layout, runs of R rows per kz
  for (int f = 0; f < sp.nact; ++f) {
    if (sp.planes) {
      const cplx<T>* src = sp.s[sp.idx[f]] + row0;
      cplx<T>* dst = stg + (size_t)f * R * NH;
      for (int q = threadIdx.x; q < R * NH; q += blockDim.x) {
        const int k = q / R, r = q % R;
        cp_async_c(dst + r * NH + k, src + (size_t)k * N * N + r, true);
      }
    } else {
      cp_async_block16(stg + (size_t)f * R * NH, sp.s[sp.idx[f]] + row0 * NH, (size_t)R * NH * sizeof(cplx<T>));
    }
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
    T po[R];                                           // P g_old, loaded ahead of the stores
    if (a.pyout) {
#pragma unroll
      for (int r = 0; r < R; ++r) po[r] = __ldg(a.pold + off + r * N + jt);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const T v = fP[r * rp + jt];
      a.out[off + r * N + jt] = v;
      if (a.pyout) a.pyout[off + r * N + jt] = v - po[r];
    }
    return;
  }
  const EpiPoint<T> ep(sp, a);
  AccShort<T> acc[8];
  // (the loads of the next row are issued before this row's stores of g')
  const T* src0 = (a.mode == 0 ? a.rho : a.psi) + off + jt;
  const T* dsrc = a.mode == 1 ? a.d + off + jt : nullptr;
  T xn = __ldg(src0), dn = dsrc ? __ldg(dsrc) : (T)0;
  for (int r = 0; r < R; ++r) {
    const int qs = r * rp + jt, q = r * N + jt;
    const T x = xn, dd = dn;
    if (r + 1 < R) { xn = __ldg(src0 + (r + 1) * N); if (dsrc) dn = __ldg(dsrc + (r + 1) * N); }
    ep.point(a, x, dd, realf[0] ? realf[0][qs] : (T)0,
             realf[1] ? realf[1][qs] : (T)0, realf[2] ? realf[2][qs] : (T)0, off + q, acc);
  }
  typename TreeVal<T>::type* scr = reinterpret_cast<typename TreeVal<T>::type*>(smem_raw);
  block_sum_tree_raw<8, T>(acc, a.partials + (size_t)blockIdx.x * 8, scr);
  if (arrive_last(a.counter)) {
    finalize_eval<T>(a.fin, scr);
    if (threadIdx.x == 0) *a.counter = 0u;
  }
}


// ---------------------------------------------------------------------------
// The y and x passes for n = 256: length-256 complex transforms of the
// columns of a 256 x 16 tile, 256 = 16 x 16, one team of 16 threads (a half
// warp) per column: thread j holds the 16 elements j + 16 s and applies a
// radix-16 butterfly, the team exchanges through shared memory, and thread j
// finishes butterfly j of the second stage with the twiddles W_256^(j r).
// The tile is staged in shared memory with a row pitch of 17 (coalesced
// loads and stores of its 16-column rows); after the first stage the tile's
// space holds the 16 teams' exchange buffers.
struct Y256 {
  static constexpr int N = 256, NH = 129, J = 16, P = J + 1, A = 16;
  static constexpr int TEAMS = 16;                     // 256 threads / 16
};

template <typename T>
__host__ __device__ constexpr size_t y256_bytes() {
  return (size_t)Y256::N * Y256::P * sizeof(cplx<T>) + (size_t)Y256::N * sizeof(cplx<T>);
}
template <typename T>
__host__ __device__ constexpr size_t x256_bytes() {
  return 2 * (size_t)Y256::N * Y256::P * sizeof(cplx<T>) + (size_t)Y256::N * sizeof(cplx<T>);
}

// v[s] = column c's elements j + 16 s of the tile (pitch 17)
template <typename T>
__device__ __forceinline__ void t256_load(const cplx<T>* tile, int c, int j, cplx<T> (&v)[16]) {
#pragma unroll
  for (int s = 0; s < 16; ++s) v[s] = tile[(j + 16 * s) * Y256::P + c];
}

// The rest of a team's transform after the radix-16 butterflies of stage 1
// on v (element order as loaded): exchange through xb (this team's 272
// slots; the caller has ordered any earlier use of them), stage 2 with the
// twiddles W_256^(j r) (conjugated for DIR > 0).  On return v[r] holds the
// result's element j + 16 r.
// The team is one half warp: its barrier names only its own 16 lanes (the
// other half's team may be idle).
__device__ __forceinline__ unsigned half_warp_mask() { return 0xFFFFu << (threadIdx.x & 16); }

template <typename T, int DIR>
__device__ __forceinline__ void t256_stage2(cplx<T>* xb, const cplx<T>* __restrict__ tw, int j, cplx<T> (&v)[16]) {
#pragma unroll
  for (int s = 0; s < 16; ++s) xb[j * 17 + s] = v[s];              // y[16 j + s] at 17 j + s
  __syncwarp(half_warp_mask());
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = xb[j + 17 * r];              // y[j + 16 r]
#pragma unroll
  for (int r = 1; r < 16; ++r) {
    cplx<T> w = tw[j * r];
    if (DIR > 0) w.y = -w.y;
    v[r] = cmul(v[r], w);
  }
  Codelet<cplx<T>, 16, DIR>::run(v);
}

// The G-space terms at one wave vector (m^2 = |m|^2, Hermitian weight w) of
// field fid's transform F (unnormalised): the output spectrum and the energy
// sums acc (0 E_H, 1 E_loc, 2 E_NL, 3 E_vW raw), as in k_xgspace.  vloc()
// returns V_loc(G) where |G|^2 <= the cutoff (called only there).
template <typename T, typename VL>
__device__ __forceinline__ cplx<T> gspace_point(int fid, const GArgs<T>& g, int merged, bool with_loc, int m2, T w,
                                                cplx<T> F, VL&& vloc, AccShort<T> (&acc)[4]) {
  const T G2 = g.tp2 * (T)m2;
  const T vr = F.x * g.invN, vi = F.y * g.invN;        // f~(G)
  const T a2 = vr * vr + vi * vi;
  if (fid == 0) {
    T orr = 0, oi = 0;
    if (g.hartree && m2 > 0) {
      const T cc = (T)(4.0 * kPi) / G2;
      acc[0].add(w * g.halfOm * cc * a2);
      orr = cc * vr; oi = cc * vi;
    }
    if (with_loc && G2 <= g.g2cut_loc) {
      const cplx<T> vl = vloc();
      acc[1].add(w * g.Om * (vr * vl.x + vi * vl.y));
      orr += vl.x; oi += vl.y;
    }
    return mk<T>(orr, oi);
  }
  if (fid == 1) {
    const T k = g.K[m2];
    acc[2].add(w * g.Om * k * a2);
    return mk<T>(k * vr, k * vi);
  }
  if (g.prec != nullptr) {
    const T pg = g.prec[m2];
    return mk<T>(pg * vr, pg * vi);
  }
  acc[3].add(w * g.halfOm * G2 * a2);
  if (merged) {
    const T k = g.K[m2];
    acc[2].add(w * g.Om * k * a2);
    const T cc = k + (T)0.5 * G2;
    return mk<T>(cc * vr, cc * vi);
  }
  return mk<T>(G2 * vr, G2 * vi);
}

// 2./4. FFT along y for n = 256, in place.  grid.x = 256 x-rows x 9 kz tiles
// of 16 (the last holds kz = 128 only), grid.y = active field.
template <typename T, int DIR>
__global__ void __launch_bounds__(256, 3) k_ypass256(Spectra<T> sp, const cplx<T>* __restrict__ tw_n) {
  constexpr int N = Y256::N, NH = Y256::NH, J = Y256::J, P = Y256::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tile = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tw = tile + N * P;
  constexpr int ntz = (NH + J - 1) / J;
  const int x = blockIdx.x / ntz, kz0 = (blockIdx.x % ntz) * J;
  const int jn = min(J, NH - kz0);
  cplx<T>* base = sp.s[sp.idx[blockIdx.y]] + (size_t)x * N * NH + kz0;
  for (int q = threadIdx.x; q < N * J; q += blockDim.x) {
    const int y = q >> 4, c = q & 15;
    if (c < jn) cp_async_c(tile + y * P + c, base + y * NH + c, true);
  }
  cp_async_commit();
  tw[threadIdx.x] = tw_n[threadIdx.x];
  cp_async_wait<0>();
  __syncthreads();
  const int c = threadIdx.x >> 4, j = threadIdx.x & 15;
  const bool act = c < jn;
  cplx<T> v[16];
  if (act) {
    t256_load<T>(tile, c, j, v);
    Codelet<cplx<T>, 16, DIR>::run(v);
  }
  __syncthreads();                                     // the tile becomes exchange space
  if (act) t256_stage2<T, DIR>(tile + c * 272, tw, j, v);
  __syncthreads();
  if (act) {
#pragma unroll
    for (int r = 0; r < 16; ++r) tile[(j + 16 * r) * P + c] = v[r];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < N * J; q += blockDim.x) {
    const int y = q >> 4, c2 = q & 15;
    if (c2 < jn) base[y * NH + c2] = tile[y * P + c2];
  }
}

// 3. FFT along x, the G-space terms, inverse FFT along x for n = 256.  Tile:
// the 256 kx of 16 consecutive flattened (ky, kz) columns; grid.x = 256 * 129
// / 16 tiles, grid.y = active field.  The forward result of thread j (kx =
// j + 16 r) is exactly the set the inverse's first stage needs, so the
// inverse starts in registers.  Same G-space arithmetic as k_xgspace.
// smem: tile[256][17] | vtile[256][17] (V_loc, field 0) | tw[256].
template <typename T>
__global__ void __launch_bounds__(256, 3) k_xgspace256(Spectra<T> sp, GArgs<T> g, const cplx<T>* __restrict__ tw_n) {
  constexpr int N = Y256::N, NH = Y256::NH, J = Y256::J, P = Y256::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tile = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* vtile = tile + N * P;
  cplx<T>* tw = vtile + N * P;
  constexpr size_t plane = (size_t)N * NH;             // stride between consecutive kx
  const size_t j0 = (size_t)blockIdx.x * J;            // N * NH is a multiple of 16
  const int fid = sp.idx[blockIdx.y];
  const bool with_loc = fid == 0 && g.vloc != nullptr;
  const T tp2 = g.tp2;
  const T g2cut = g.g2cut_loc;
  cplx<T>* base = sp.s[fid] + j0;
  for (int q = threadIdx.x; q < N * J; q += blockDim.x) {
    const int kx = q >> 4, jc = q & 15;
    cp_async_c(tile + kx * P + jc, base + kx * plane + jc, true);
    if (with_loc) {
      const int jl = (int)j0 + jc;
      const int ky = jl / NH, kz = jl - ky * NH;
      const int mx = kx <= 127 ? kx : kx - N, my = ky <= 127 ? ky : ky - N;
      const bool need = tp2 * (T)(mx * mx + my * my + kz * kz) <= g2cut;
      cp_async_c(vtile + kx * P + jc, g.vloc + (need ? kx * plane + j0 + jc : 0), need);
    }
  }
  cp_async_commit();
  tw[threadIdx.x] = tw_n[threadIdx.x];
  cp_async_wait<0>();
  __syncthreads();
  const int c = threadIdx.x >> 4, j = threadIdx.x & 15;
  cplx<T> v[16];
  t256_load<T>(tile, c, j, v);
  Codelet<cplx<T>, 16, -1>::run(v);
  __syncthreads();                                     // the tile becomes exchange space
  cplx<T>* xb = tile + c * 272;
  t256_stage2<T, -1>(xb, tw, j, v);                    // v[r] = F(kx = j + 16 r)
  // G-space terms of column (ky, kz)
  const int jl = (int)j0 + c;
  const int ky = jl / NH, kz = jl - ky * NH;
  const int my = ky <= 127 ? ky : ky - N;
  const T w = (kz == 0 || kz == 128) ? (T)1 : (T)2;
  AccShort<T> acc[4];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int kx = j + 16 * r;
    const int mx = kx <= 127 ? kx : kx - N;
    const int m2 = mx * mx + my * my + kz * kz;
    v[r] = gspace_point<T>(fid, g, sp.merged, with_loc, m2, w, v[r], [&]() { return vtile[kx * P + c]; }, acc);
  }
  // inverse along kx: stage 1 on the elements j + 16 r already held
  Codelet<cplx<T>, 16, +1>::run(v);
  __syncwarp(half_warp_mask());                        // the team's reads of xb are done
  t256_stage2<T, +1>(xb, tw, j, v);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) tile[(j + 16 * r) * P + c] = v[r];
  __syncthreads();
  for (int q = threadIdx.x; q < N * J; q += blockDim.x) {
    const int kx = q >> 4, jc = q & 15;
    base[kx * plane + jc] = tile[kx * P + jc];
  }
  const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
  block_sum_tree_raw<4, T>(acc, g.partials + b * 4, reinterpret_cast<typename TreeVal<T>::type*>(smem_raw));
}

// ---------------------------------------------------------------------------
// The x-y transforms and the G-space terms of one kz plane of one field in a
// cluster of eight blocks (plane layout, [kz][x][y]).  A 256 x 256 FP32 plane
// (512 KB) fits no block's shared memory; block c of the cluster keeps the 32
// rows x = 8 b + c (b = 0..31, unpadded: every access below has a warp's
// lanes along a row, or at exchange slots that differ in bank).  The
// transform along x splits as 256 = 32 x 8 (four-step):
//   X[k2 + 32 k1] = sum_c W_8^(c k1) [W_256^(c k2) sum_b W_32^(b k2) x[8 b + c]],
// so each block does the inner 32-point transforms of its own rows, and only
// the outer 8-point transforms (one per (k2, ky)) combine the blocks:
//   1. forward transforms along y of its 32 rows;
//   2. forward 32-point transforms along b of its 256 columns, times
//      W_256^(c k2) (all local);
//   -- cluster barrier --
//   3. for its k2 = 4 c .. 4 c + 3 and every ky: the eight values (one per
//      block, same offset: a warp reads 256 contiguous bytes of each) through
//      distributed shared memory, the 8-point transform, the G-space terms at
//      kx = k2 + 32 k1, the inverse 8-point transform, the values back;
//   -- cluster barrier --
//   4. times W_256^(-c k2), inverse 32-point transforms along k2; inverse
//      transforms along y of its rows; the rows back to memory.
// Two cluster barriers in all.  The y transforms keep the y pass's
// butterflies exactly (half-warp teams, 256 = 16 x 16, the exchange in place
// in the row); the x transforms group the same sums differently (32 x 8 in
// place of 16 x 16), so results agree with the other passes to FP32 rounding.
// grid = (8 * 129 kz, active field), 256 threads, 66 KB of shared memory
// (slice[32][256] | tw[256]): up to three blocks per SM.  FP32 only (the
// row copies move two complex values per 16 bytes).
struct P256 {
  static constexpr int N = 256, NH = 129, CL = 8, ROWS = N / CL, P = N, THREADS = 256;
};

template <typename T>
__host__ __device__ constexpr size_t p256_bytes() {
  return ((size_t)P256::ROWS * P256::P + P256::N) * sizeof(cplx<T>);
}

// A half-warp team's length-256 transform of one row (256 = 16 x 16, the
// butterflies of t256_stage2), in place: the exchange between the two
// stages goes through the row itself, element e at
// 16 (e / 16) + (e + e / 16) % 16 (the 16 lanes hit 16 different bank pairs
// in both exchange patterns).
template <typename T, int DIR>
__device__ __forceinline__ void p256_row(cplx<T>* row, const cplx<T>* __restrict__ tw, int j) {
  const unsigned mask = half_warp_mask();
  cplx<T> v[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) v[s] = row[j + 16 * s];
  Codelet<cplx<T>, 16, DIR>::run(v);
  __syncwarp(mask);                                    // the team has read the row
#pragma unroll
  for (int s = 0; s < 16; ++s) row[16 * j + ((s + j) & 15)] = v[s];   // y[16 j + s]
  __syncwarp(mask);
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = row[16 * r + ((j + r) & 15)];   // y[j + 16 r]
#pragma unroll
  for (int r = 1; r < 16; ++r) {
    cplx<T> w = tw[j * r];
    if (DIR > 0) w.y = -w.y;
    v[r] = cmul(v[r], w);
  }
  Codelet<cplx<T>, 16, DIR>::run(v);
  __syncwarp(mask);                                    // the team has read the exchange
#pragma unroll
  for (int r = 0; r < 16; ++r) row[j + 16 * r] = v[r];
}

// Length-32 transform of v in registers, natural order in and out: one
// radix-2 step (x_i +- x_(i+16), the difference times W_32^i = tw[8 i]), then
// 16-point transforms of the two halves (even and odd outputs).
template <typename T, int DIR>
__device__ __forceinline__ void p256_dft32(cplx<T> (&v)[32], const cplx<T>* __restrict__ tw) {
  cplx<T> u[16], d[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    u[i] = cadd(v[i], v[i + 16]);
    d[i] = csub(v[i], v[i + 16]);
    if (i > 0) {
      cplx<T> w = tw[8 * i];
      if (DIR > 0) w.y = -w.y;
      d[i] = cmul(d[i], w);
    }
  }
  Codelet<cplx<T>, 16, DIR>::run(u);
  Codelet<cplx<T>, 16, DIR>::run(d);
#pragma unroll
  for (int k = 0; k < 16; ++k) { v[2 * k] = u[k]; v[2 * k + 1] = d[k]; }
}

template <typename T>
__global__ void __cluster_dims__(8, 1, 1) __launch_bounds__(256, 3)
k_plane256cl(Spectra<T> sp, GArgs<T> g, const cplx<T>* __restrict__ tw_n) {
  static_assert(sizeof(T) == 4, "FP32 plans only");
  namespace cg = cooperative_groups;
  constexpr int N = P256::N, ROWS = P256::ROWS, P = P256::P, CL = P256::CL;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* slice = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tw = slice + ROWS * P;
  const int c = (int)cl.block_rank();
  const int kz = blockIdx.x / CL;
  const int fid = sp.idx[blockIdx.y];
  cplx<T>* gpl = sp.s[fid] + (size_t)kz * N * N + (size_t)c * N;   // row x = 8 b + c at gpl + 8 b N
  for (int q = threadIdx.x; q < ROWS * N / 2; q += blockDim.x) {   // 16-byte pieces
    const int b = q >> 7, y = (q & 127) * 2;
    cp_async<16>(slice + b * P + y, gpl + (size_t)b * CL * N + y, true);
  }
  cp_async_commit();
  tw[threadIdx.x] = tw_n[threadIdx.x];
  cp_async_wait<0>();
  __syncthreads();
  const int team = threadIdx.x >> 4, j = threadIdx.x & 15, t = threadIdx.x;
  // 1. along y
  for (int b0 = 0; b0 < ROWS; b0 += 16) p256_row<T, -1>(slice + (b0 + team) * P, tw, j);
  __syncthreads();
  // 2. column ky = t: 32-point transforms along b, twiddles W_256^(c k2)
  {
    cplx<T> v[32];
#pragma unroll
    for (int b = 0; b < 32; ++b) v[b] = slice[b * P + t];
    p256_dft32<T, -1>(v, tw);
#pragma unroll
    for (int k2 = 1; k2 < 32; ++k2) v[k2] = cmul(v[k2], tw[c * k2]);
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) slice[k2 * P + t] = v[k2];
  }
  cl.sync();
  // 3. across the cluster: the (k2, ky = t) sums of the eight blocks
  cplx<T>* part[CL];
#pragma unroll
  for (int o = 0; o < CL; ++o) part[o] = cl.map_shared_rank(slice, o);
  const bool with_loc = fid == 0 && g.vloc != nullptr;
  const T w = (kz == 0 || kz == N / 2) ? (T)1 : (T)2;
  const int my = t <= 127 ? t : t - N;
  AccShort<T> acc[4];
  for (int i = 0; i < 4; ++i) {
    const int k2 = 4 * c + i;
    cplx<T> z[CL];
#pragma unroll
    for (int o = 0; o < CL; ++o) z[o] = part[o][k2 * P + t];
    Codelet<cplx<T>, 8, -1>::run(z);                   // z[k1] = F(kx = k2 + 32 k1)
    // V_loc in plane layout [kz][kx][ky]
    const cplx<T>* vl = with_loc ? g.vloc + (size_t)kz * N * N + t : nullptr;
#pragma unroll
    for (int k1 = 0; k1 < CL; ++k1) {
      const int kx = k2 + 32 * k1;
      const int mx = kx <= 127 ? kx : kx - N;
      const int m2 = mx * mx + my * my + kz * kz;
      z[k1] = gspace_point<T>(fid, g, sp.merged, with_loc, m2, w, z[k1], [&]() { return vl[(size_t)kx * N]; }, acc);
    }
    Codelet<cplx<T>, 8, +1>::run(z);
#pragma unroll
    for (int o = 0; o < CL; ++o) part[o][k2 * P + t] = z[o];
  }
  cl.sync();                                           // (no remote access after this)
  // 4. column ky = t: twiddles W_256^(-c k2), inverse 32-point transforms
  {
    cplx<T> v[32];
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) v[k2] = slice[k2 * P + t];
#pragma unroll
    for (int k2 = 1; k2 < 32; ++k2) v[k2] = cmul(v[k2], cconj(tw[c * k2]));
    p256_dft32<T, 1>(v, tw);
#pragma unroll
    for (int b = 0; b < 32; ++b) slice[b * P + t] = v[b];
  }
  __syncthreads();
  for (int b0 = 0; b0 < ROWS; b0 += 16) p256_row<T, 1>(slice + (b0 + team) * P, tw, j);
  __syncthreads();
  for (int q = threadIdx.x; q < ROWS * N / 2; q += blockDim.x) {
    const int b = q >> 7, y = (q & 127) * 2;
    *reinterpret_cast<float4*>(gpl + (size_t)b * CL * N + y) = *reinterpret_cast<const float4*>(slice + b * P + y);
  }
  const size_t bi = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
  block_sum_tree_raw<4, T>(acc, g.partials + bi * 4, reinterpret_cast<typename TreeVal<T>::type*>(smem_raw));
}

// One-time reorder of V_loc from the tiled layout [kx][ky][kz] into plane
// layout, natural order: dst[(kz 256 + kx) 256 + ky] = src[(kx 256 + ky) 129 + kz].
template <typename T>
__global__ void k_vloc_planes256(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst) {
  constexpr int N = 256, NH = 129;
  const size_t tot = (size_t)NH * N * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)(i % N);
    const int kx = (int)((i / N) % N);
    const int kz = (int)(i / ((size_t)N * N));
    dst[i] = src[((size_t)kx * N + ky) * NH + kz];
  }
}

}  // namespace ofdft
