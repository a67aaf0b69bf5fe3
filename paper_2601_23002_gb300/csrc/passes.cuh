// The per-evaluation kernels of the functional (templated on the real type T).
//
// One evaluation of F[n] and its potential is five launches over the grid:
//   1. k_zfwd      prologue (n, n^a, psi from rho or from psi + t d) fused with
//                  the real-to-complex FFT along z (a half-length complex FFT
//                  per row for even n, one length-n complex FFT per two rows
//                  for odd n).
//   2. k_ypass<-1> complex FFT along y.
//   3. k_xgspace   FFT along x, every G-space term (Hartree + local
//                  pseudopotential, nonlocal kernel K(|G|), vW |G|^2) with its
//                  FP64 energy partial sums, inverse FFT along x.
//   4. k_ypass<+1> inverse FFT along y.
//   5. k_zinv_epi  complex-to-real FFT along z fused with the pointwise
//                  functional (finite-T TF through the inverse Fermi-Dirac
//                  integral, PZ LDA XC, v_NL) and the potential / gradient.
// plus k_finalize, a one-block FP64 reduction of the per-block partial sums.
//
// Layouts: real fields [n][n][n] (z fastest); half spectra [n][n][n/2+1].
#pragma once
#include "common.cuh"
#include "fft.cuh"
#include "fd_fit_tables.h"

namespace ofdft {

constexpr double kNmin = 1e-20;        // density floor in powers and logarithms
constexpr double kPhiMin = 1e-10;      // sqrt(n) floor in the vW potential

enum : int { FIELD_N = 1, FIELD_NA = 2, FIELD_PSI = 4 };

template <typename T> struct Spectra {
  cplx<T>* s[3];    // by field index 0 = n, 1 = n^a, 2 = psi
  int nact;         // number of active fields
  int idx[3];       // active field indices, in order
  // merged = 1 when a = 1/2 with both vW and NL on: n^(1/2) = sqrt(scale) psi,
  // so field 2 carries both terms: W = IFFT[(K + G^2/2) psi~] and
  // psi v_NL + (-lap psi)/2 = W (for psi >= 0); field 1 is not used
  int merged;
  // layout of the half spectra: 0 = tiled [kx][ky][kz]; 1 = plane [kz][kx][ky]
  // (entry (kz, x, y) at kz n^2 + x n + y, i.e. kz n^2 + real-space row)
  int planes;
};

// ---------------------------------------------------------------------------
// Finite-temperature Thomas-Fermi pointwise: eta(y) and p(y) from the
// piecewise Chebyshev tables (see gen_fd_fits.py); f_TF = n T (eta - p),
// v_TF = T eta.
static __device__ __forceinline__ void fd_eta_p(double y, double& eta, double& p) {
  const double s = log(y);
  const double lngamma32 = -0.12078223763524522234551844578164;  // ln Gamma(3/2)
  if (s < FD_S_LO) {
    const double u = y * 1.1283791670955125738961589031215;      // y / Gamma(3/2)
    eta = s - lngamma32 + u * 0.35355339059327376220042218105242;   // + u / 2^(3/2)
    p = 1.0 + u * 0.17677669529663688110021109052621;               // 1 + u / 2^(5/2)
  } else if (s >= FD_S_HI) {
    const double e0 = pow(1.5 * y, 2.0 / 3.0);
    eta = e0 * (1.0 - 0.82246703342411321823620758332301 / (e0 * e0));   // pi^2/12
    p = 0.4 * eta * (1.0 + 4.9348022005446793094172454999381 / (eta * eta));  // pi^2/2
  } else {
    const double r = (s - FD_S_LO) / FD64_W;
    int i = (int)r;
    i = i < 0 ? 0 : (i >= FD64_NINT ? FD64_NINT - 1 : i);
    const double x = 2.0 * (r - (double)i) - 1.0;
    double ce[FD64_NC], cp[FD64_NC];
    static_assert(FD64_NC % 2 == 0, "16-byte loads");
    const double2* e2 = reinterpret_cast<const double2*>(fd64_eta[i]);
    const double2* p2 = reinterpret_cast<const double2*>(fd64_p[i]);
#pragma unroll
    for (int k = 0; k < FD64_NC / 2; ++k) {
      const double2 ev = __ldg(e2 + k), pv = __ldg(p2 + k);
      ce[2 * k] = ev.x; ce[2 * k + 1] = ev.y; cp[2 * k] = pv.x; cp[2 * k + 1] = pv.y;
    }
    double b1 = 0, b2 = 0, c1 = 0, c2 = 0;
#pragma unroll
    for (int k = FD64_NC - 1; k >= 1; --k) {
      const double t = fma(2.0 * x, b1, ce[k] - b2); b2 = b1; b1 = t;
      const double u = fma(2.0 * x, c1, cp[k] - c2); c2 = c1; c1 = u;
    }
    eta = fma(x, b1, ce[0] - b2);
    p = fma(x, c1, cp[0] - c2);
  }
}

static __device__ __forceinline__ void fd_eta_p(float y, float& eta, float& p) {
  const float s = __logf(y);      // a few ulp: far below the fit's use of s
  const float lngamma32 = -0.120782237635245222f;
  if (s < (float)FD_S_LO) {
    const float u = y * 1.12837916709551257f;
    eta = s - lngamma32 + u * 0.353553390593273762f;
    p = 1.0f + u * 0.176776695296636881f;
  } else if (s >= (float)FD_S_HI) {
    const float e0 = powf(1.5f * y, 2.0f / 3.0f);
    eta = e0 * (1.0f - 0.822467033424113218f / (e0 * e0));
    p = 0.4f * eta * (1.0f + 4.93480220054467931f / (eta * eta));
  } else {
    const float r = (s - (float)FD_S_LO) * (1.0f / FD32_W);
    int i = (int)r;
    i = i < 0 ? 0 : (i >= FD32_NINT ? FD32_NINT - 1 : i);
    const float x = 2.0f * (r - (float)i) - 1.0f;
    // each interval's 8 coefficients as two 16-byte loads per table
    float ce[FD32_NC], cp[FD32_NC];
    static_assert(FD32_NC == 8, "two float4 per interval");
    const float4* e4 = reinterpret_cast<const float4*>(fd32_eta[i]);
    const float4* p4 = reinterpret_cast<const float4*>(fd32_p[i]);
    const float4 ea = __ldg(e4), eb = __ldg(e4 + 1), pa = __ldg(p4), pb = __ldg(p4 + 1);
    ce[0] = ea.x; ce[1] = ea.y; ce[2] = ea.z; ce[3] = ea.w; ce[4] = eb.x; ce[5] = eb.y; ce[6] = eb.z; ce[7] = eb.w;
    cp[0] = pa.x; cp[1] = pa.y; cp[2] = pa.z; cp[3] = pa.w; cp[4] = pb.x; cp[5] = pb.y; cp[6] = pb.z; cp[7] = pb.w;
    float b1 = 0, b2 = 0, c1 = 0, c2 = 0;
#pragma unroll
    for (int k = FD32_NC - 1; k >= 1; --k) {
      const float t = fmaf(2.0f * x, b1, ce[k] - b2); b2 = b1; b1 = t;
      const float u = fmaf(2.0f * x, c1, cp[k] - c2); c2 = c1; c1 = u;
    }
    eta = fmaf(x, b1, ce[0] - b2);
    p = fmaf(x, c1, cp[0] - c2);
  }
}

// Perdew-Zunger LDA, unpolarised: returns e_xc per electron, v_xc.
// PZ81 joins its two correlation branches at r_s = 1 by continuity of e_c and
// d e_c / d r_s, which fixes B and D from the other constants; the printed
// three-digit B = -0.048, D = -0.0116 are their rounding and leave a 3.2e-5 Ha
// step at r_s = 1 that stalls the minimiser on densities straddling it.
constexpr double kPzG = -0.1423, kPzB1 = 1.0529, kPzB2 = 0.3334, kPzA = 0.0311, kPzC = 0.0020;
constexpr double kPzDen1 = 1.0 + kPzB1 + kPzB2;
// A + C + D = d e_c/d r_s of the low-density branch at 1;  B + D = its e_c at 1
constexpr double kPzD = -kPzG * (0.5 * kPzB1 + kPzB2) / (kPzDen1 * kPzDen1) - kPzA - kPzC;
constexpr double kPzB = kPzG / kPzDen1 - kPzD;

template <typename T>
__device__ __forceinline__ void pz81(T n, T& exc, T& vxc) {
  const T third = (T)(1.0 / 3.0);
  const T cbn = cbrt(n);
  // r_s = (3 / (4 pi n))^(1/3)
  const T rs = (T)0.62035049089940001666800681204778 / cbn;
  const T ex = (T)-0.73855876638202240588423003268 * cbn;   // -(3/4)(3/pi)^(1/3) n^(1/3)
  const T vx = (T)(4.0 / 3.0) * ex;
  T ec, vc;
  if (rs >= (T)1) {
    const T g = (T)kPzG, b1 = (T)kPzB1, b2 = (T)kPzB2;
    const T sq = sqrt(rs);
    const T den = (T)1 + b1 * sq + b2 * rs;
    ec = g / den;
    vc = ec * ((T)1 + (T)(7.0 / 6.0) * b1 * sq + (T)(4.0 / 3.0) * b2 * rs) / den;
  } else {
    const T A = (T)kPzA, B = (T)kPzB, C = (T)kPzC, D = (T)kPzD;
    const T ln = log(rs);
    ec = A * ln + B + C * rs * ln + D * rs;
    vc = A * ln + (B - A * third) + (T)(2.0 / 3.0) * C * rs * ln + ((T)2 * D - C) * third * rs;
  }
  exc = ex + ec;
  vxc = vx + vc;
}

// FP32 plans: fast reciprocals (__fdividef, a few ulp: inside the float
// rounding of the terms they feed)
template <>
__device__ __forceinline__ void pz81<float>(float n, float& exc, float& vxc) {
  const float cbn = cbrtf(n);
  const float rs = __fdividef(0.620350490899400017f, cbn);
  const float ex = -0.738558766382022406f * cbn;
  const float vx = (4.0f / 3.0f) * ex;
  float ec, vc;
  if (rs >= 1.0f) {
    const float g = (float)kPzG, b1 = (float)kPzB1, b2 = (float)kPzB2;
    const float sq = sqrtf(rs);
    const float inv = __fdividef(1.0f, 1.0f + b1 * sq + b2 * rs);
    ec = g * inv;
    vc = ec * (1.0f + (7.0f / 6.0f) * b1 * sq + (4.0f / 3.0f) * b2 * rs) * inv;
  } else {
    const float A = (float)kPzA, B = (float)kPzB, C = (float)kPzC, D = (float)kPzD;
    const float ln = __logf(rs);
    ec = A * ln + B + C * rs * ln + D * rs;
    vc = A * ln + (B - A * (1.0f / 3.0f)) + (2.0f / 3.0f) * C * rs * ln + (2.0f * D - C) * (1.0f / 3.0f) * rs;
  }
  exc = ex + ec;
  vxc = vx + vc;
}

template <typename T> __device__ __forceinline__ T pow_t(T a, T b);
template <> __device__ __forceinline__ double pow_t<double>(double a, double b) { return pow(a, b); }
template <> __device__ __forceinline__ float pow_t<float>(float a, float b) { return exp2f(b * log2f(a)); }

// ---------------------------------------------------------------------------
// 1. prologue + R2C along z
template <typename T> struct ProArgs {
  int mode;            // 0: density rho given; 1: psi + t d with n = scale psi^2
  const T* rho;
  const T* psi;
  const T* d;
  T t, scale, alpha;   // converted on the host: no FP64 work in the kernels
  // subtracted from psi before its transform: only G = 0 changes, and the psi
  // field's G-space factors (G^2/2, K(G) with K(0) = 0) vanish there.  With the
  // mean (about sqrt(nbar / scale)) removed, the transform's rounding scales
  // with the variation of psi instead of its size; the G^2 factor of the
  // gradient amplifies that rounding, so in FP32 this lowers the gradient's
  // noise floor several times.
  T psi_shift;
  // when set, scale = dsc[0], psi_shift = dsc[1] and t = dsc[2] (a trial
  // formed on the device, see TrialScale)
  const double* dsc;
};

// Rows of one z-pass FFT buffer: even n transforms each real row as a
// half-length complex row (R rows of pitch P); odd n packs two real rows into
// one complex row of length n (ceil(R/2) rows of pitch P = n).
__host__ __device__ __forceinline__ size_t zbuf_elems(int n, int R, int P) {
  return (n & 1) ? (size_t)((R + 1) >> 1) * P : (size_t)R * P;
}

// smem: psit[R][n] (T) | dbuf[R][n] (T) | buf0 | buf1 (complex, zbuf_elems each)
// Odd n: ph is the full-length plan and tw_h the length-n twiddles.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_zfwd(ProArgs<T> a, Spectra<T> sp, FftPlan1 ph,
                                              const cplx<T>* __restrict__ tw_h,
                                              const cplx<T>* __restrict__ tw_n, int n, int R, int P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int h = n / 2, nh = h + 1;
  T* psit = reinterpret_cast<T*>(smem_raw);
  T* dbuf = psit + (size_t)R * n;
  cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw + (((size_t)2 * R * n * sizeof(T) + 15) & ~(size_t)15));
  cplx<T>* buf1 = buf0 + zbuf_elems(n, R, P);
  const size_t row0 = (size_t)blockIdx.x * R;
  R = (int)min((size_t)R, (size_t)n * n - row0);     // rows in this block
  const size_t off = row0 * n;
  const int tot = R * n;
  // all of the block's input rows in flight at once
  // (mode 1 with d == nullptr: the field is psi itself, as in the
  // preconditioning pass)
  const T* src0 = a.mode == 0 ? a.rho : a.psi;
  const bool has_d = a.mode != 0 && a.d != nullptr;
  for (int q = threadIdx.x; q < tot; q += blockDim.x) {
    cp_async<sizeof(T)>(psit + q, src0 + off + q, true);
    if (has_d) cp_async<sizeof(T)>(dbuf + q, a.d + off + q, true);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  // psi_t (or sqrt rho) in place; the raw density stays in dbuf for mode 0
  const T tstep = a.dsc ? (T)a.dsc[2] : a.t;
  for (int q = threadIdx.x; q < tot; q += blockDim.x) {
    const T x = psit[q];
    if (a.mode == 0) { dbuf[q] = x; psit[q] = sqrt(fmax(x, (T)0)); }
    else if (has_d) psit[q] = x + tstep * dbuf[q];
  }
  __syncthreads();
  const T scale = a.dsc ? (T)a.dsc[0] : a.scale, alpha = a.alpha, nmin = (T)kNmin;
  const T psi_shift = a.dsc ? (T)a.dsc[1] : a.psi_shift;
  const unsigned Mh = qmagic(h), Mnh = qmagic(nh), MR = qmagic(R);
  const size_t nn = (size_t)n * n;
  for (int f = 0; f < sp.nact; ++f) {
    const int fid = sp.idx[f];
    if (n & 1) {
      // odd n: rows 2p and 2p + 1 as the real and imaginary parts of one
      // length-n complex row z = x_a + i x_b; with Z = FFT(z),
      //   X_a[k] = (Z[k] + Z*[n-k]) / 2,   X_b[k] = -i (Z[k] - Z*[n-k]) / 2
      auto fv = [&](int i) -> T {       // field fid at buffer position i
        const T x = psit[i];
        if (fid == 2) return x - psi_shift;
        const T nv = a.mode == 0 ? dbuf[i] : scale * x * x;
        return fid == 0 ? nv : pow_t<T>(fmax(nv, nmin), alpha);
      };
      const int npair = (R + 1) >> 1;
      const unsigned Mn = qmagic(n);
      for (int q = threadIdx.x; q < npair * n; q += blockDim.x) {
        const int pr = qdiv(q, n, Mn), j = q - pr * n;
        const int rb = 2 * pr + 1;
        buf0[pr * P + j] = mk<T>(fv(2 * pr * n + j), rb < R ? fv(rb * n + j) : (T)0);
      }
      __syncthreads();
      cplx<T>* Z = fft_smem<T, -1>(buf0, buf1, ph, 1, P, npair, tw_h);
      cplx<T>* out = sp.s[fid];
      for (int q = threadIdx.x; q < R * nh; q += blockDim.x) {
        int r, k;
        if (sp.planes) { k = qdiv(q, R, MR); r = q - k * R; }
        else { r = qdiv(q, nh, Mnh); k = q - r * nh; }
        const cplx<T>* zr = Z + (r >> 1) * P;
        const cplx<T> zk = zr[k];
        const cplx<T> zc = cconj(zr[k == 0 ? 0 : n - k]);
        cplx<T> o;
        if ((r & 1) == 0) {
          o = mk<T>((T)0.5 * (zk.x + zc.x), (T)0.5 * (zk.y + zc.y));
        } else {
          const cplx<T> dd = csub(zk, zc);
          o = mk<T>((T)0.5 * dd.y, (T)-0.5 * dd.x);
        }
        const size_t at = sp.planes ? (size_t)k * nn + row0 + r : (row0 + r) * nh + k;
        out[at] = o;
      }
      __syncthreads();
      continue;
    }
    for (int q = threadIdx.x; q < R * h; q += blockDim.x) {
      const int r = qdiv(q, h, Mh), k = q - r * h;
      T x0 = psit[r * n + 2 * k], x1 = psit[r * n + 2 * k + 1];
      if (fid == 2) { x0 -= psi_shift; x1 -= psi_shift; }
      if (fid == 0) {
        if (a.mode == 0) { x0 = dbuf[r * n + 2 * k]; x1 = dbuf[r * n + 2 * k + 1]; }
        else { x0 = scale * x0 * x0; x1 = scale * x1 * x1; }
      } else if (fid == 1) {
        T n0, n1;
        if (a.mode == 0) { n0 = dbuf[r * n + 2 * k]; n1 = dbuf[r * n + 2 * k + 1]; }
        else { n0 = scale * x0 * x0; n1 = scale * x1 * x1; }
        x0 = pow_t<T>(fmax(n0, nmin), alpha);
        x1 = pow_t<T>(fmax(n1, nmin), alpha);
      }
      buf0[r * P + k] = mk<T>(x0, x1);
    }
    __syncthreads();
    cplx<T>* Z = fft_smem<T, -1>(buf0, buf1, ph, 1, P, R, tw_h);
    // X[k] = (Z[k] + Z*[h-k])/2 - (i/2) W^k (Z[k] - Z*[h-k]),  k = 0..h
    // (plane layout: consecutive threads take consecutive rows of one kz, so
    // the block's stores form runs of R)
    cplx<T>* out = sp.s[fid];
    for (int q = threadIdx.x; q < R * nh; q += blockDim.x) {
      int r, k;
      if (sp.planes) { k = qdiv(q, R, MR); r = q - k * R; }
      else { r = qdiv(q, nh, Mnh); k = q - r * nh; }
      const cplx<T> zk = Z[r * P + (k == h ? 0 : k)];
      const cplx<T> zc = cconj(Z[r * P + (k == 0 ? 0 : h - k)]);
      const cplx<T> e = cadd(zk, zc);
      const cplx<T> o = csub(zk, zc);
      const cplx<T> w = tw_n[k];
      const cplx<T> wo = cmul(w, o);
      // -(i/2) wo = (wo.y/2, -wo.x/2)
      const size_t at = sp.planes ? (size_t)k * nn + row0 + r : (row0 + r) * nh + k;
      out[at] = mk<T>((T)0.5 * (e.x + wo.y), (T)0.5 * (e.y - wo.x));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// 2./4. FFT along y, in place.  Tile: all n values of y times J consecutive kz
// at one x.  grid.x = n * ceil(nh / J), grid.y = active field.
// smem: buf0[n][J] | buf1[n][J]
template <typename T, int DIR>
__global__ void __launch_bounds__(256, 4) k_ypass(Spectra<T> sp, FftPlan1 pn, const cplx<T>* __restrict__ tw_n,
                                               int n, int J) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* buf1 = buf0 + (size_t)n * J;
  const int nh = n / 2 + 1;
  const int ntz = (nh + J - 1) / J;
  const int x = blockIdx.x / ntz, tz = blockIdx.x % ntz;
  const int kz0 = tz * J;
  const int jn = min(J, nh - kz0);
  cplx<T>* base = sp.s[sp.idx[blockIdx.y]] + (size_t)x * n * nh + kz0;
  const int lgJ = __ffs(J) - 1;              // J is a power of two
  for (int q = threadIdx.x; q < n * J; q += blockDim.x) {
    const int y = q >> lgJ, j = q & (J - 1);
    cp_async_c(buf0 + q, base + (j < jn ? (size_t)y * nh + j : 0), j < jn);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  cplx<T>* res = fft_smem<T, DIR>(buf0, buf1, pn, J, 1, J, tw_n);
  for (int q = threadIdx.x; q < n * J; q += blockDim.x) {
    const int y = q >> lgJ, j = q & (J - 1);
    if (j < jn) base[(size_t)y * nh + j] = res[q];
  }
}

// FFT along x only (no G-space work), in place; used for analysis transforms.
template <typename T, int DIR>
__global__ void __launch_bounds__(256, 4) k_xpass(Spectra<T> sp, FftPlan1 pn, const cplx<T>* __restrict__ tw_n,
                                               int n, int J) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* buf1 = buf0 + (size_t)n * J;
  const int nh = n / 2 + 1;
  const size_t plane = (size_t)n * nh;
  const size_t j0 = (size_t)blockIdx.x * J;
  const int jn = (int)min((size_t)J, plane - j0);
  cplx<T>* base = sp.s[sp.idx[blockIdx.y]] + j0;
  const int lgJ = __ffs(J) - 1;              // J is a power of two
  for (int q = threadIdx.x; q < n * J; q += blockDim.x) {
    const int kx = q >> lgJ, j = q & (J - 1);
    cp_async_c(buf0 + q, base + (j < jn ? (size_t)kx * plane + j : 0), j < jn);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  cplx<T>* res = fft_smem<T, DIR>(buf0, buf1, pn, J, 1, J, tw_n);
  for (int q = threadIdx.x; q < n * J; q += blockDim.x) {
    const int kx = q >> lgJ, j = q & (J - 1);
    if (j < jn) base[(size_t)kx * plane + j] = res[q];
  }
}

// ---------------------------------------------------------------------------
// 3. FFT along x + G-space terms + inverse FFT along x.
// Tile: all n values of kx times J consecutive flattened (ky, kz).
template <typename T> struct GArgs {
  const cplx<T>* vloc;   // V_loc(G), half spectrum (may be null: no local term)
  const T* K;            // K(m^2) table
  T tp2;                 // (2 pi / L)^2
  T Om, halfOm, invN;    // Omega, Omega/2, 1/N
  T g2cut_loc;           // V_loc negligible beyond this |G|^2
  int hartree;           // 1: add 4 pi n~/G^2 to the n field
  // [gridDim.y * gridDim.x][4]: E_H, E_loc, E_NL, E_vW(raw), as float-float
  // pairs (FP32 plans) or doubles
  typename TreeVal<T>::type* partials;
  // non-null: the psi field is the minimiser's preconditioning pass, and its
  // spectrum is multiplied by this table of p(m^2) instead (see minimize)
  const T* prec;
};

// One block per (tile, field): blockIdx.y indexes the active fields.
// smem: buf0[n][J] | buf1[n][J] | vbuf[n][J] (V_loc tile, field 0 only)
template <typename T>
__global__ void __launch_bounds__(256) k_xgspace(Spectra<T> sp, GArgs<T> g, FftPlan1 pn,
                                                 const cplx<T>* __restrict__ tw_n, int n, int J) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* buf1 = buf0 + (size_t)n * J;
  cplx<T>* vbuf = buf1 + (size_t)n * J;
  const int nh = n / 2 + 1;
  const size_t plane = (size_t)n * nh;   // stride between consecutive kx
  const size_t j0 = (size_t)blockIdx.x * J;
  const int jn = (int)min((size_t)J, plane - j0);
  // G-space arithmetic in the plan's precision (float for FP32 plans)
  const T tp2 = g.tp2, invN = g.invN, Om = g.Om, halfOm = g.halfOm, fourpi = (T)(4.0 * kPi);
  const T g2cut = g.g2cut_loc;
  const int lgJ = __ffs(J) - 1;              // J is a power of two
  const unsigned Mnh = qmagic(nh);
  const int fid = sp.idx[blockIdx.y];
  const bool with_loc = fid == 0 && g.vloc != nullptr;
  AccShort<T> acc[4];
  cplx<T>* base = sp.s[fid] + j0;
  // the block's spectrum tile and (field 0) its V_loc entries inside the cutoff, all in flight
  for (int q = threadIdx.x; q < n * J; q += blockDim.x) {
    const int kx = q >> lgJ, j = q & (J - 1);
    const bool in = j < jn;
    cp_async_c(buf0 + q, base + (in ? (size_t)kx * plane + j : 0), in);
    if (with_loc) {
      bool need = false;
      if (in) {
        const int jl = (int)(j0 + j);
        const int ky = qdiv(jl, nh, Mnh), kz = jl - ky * nh;
        const int mx = kx <= (n - 1) / 2 ? kx : kx - n;
        const int my = ky <= (n - 1) / 2 ? ky : ky - n;
        need = tp2 * (T)(mx * mx + my * my + kz * kz) <= g2cut;
      }
      cp_async_c(vbuf + q, g.vloc + (need ? (size_t)kx * plane + j0 + j : 0), need);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  cplx<T>* F = fft_smem<T, -1>(buf0, buf1, pn, J, 1, J, tw_n);
  for (int q = threadIdx.x; q < n * J; q += blockDim.x) {
    const int kx = q >> lgJ, j = q & (J - 1);
    if (j >= jn) { F[q] = mk<T>(0, 0); continue; }
    const int jl = (int)(j0 + j);                 // < n (n/2+1) <= 2^17
    const int ky = qdiv(jl, nh, Mnh), kz = jl - ky * nh;
    const int mx = kx <= (n - 1) / 2 ? kx : kx - n;
    const int my = ky <= (n - 1) / 2 ? ky : ky - n;
    const int m2 = mx * mx + my * my + kz * kz;
    const T G2 = tp2 * (T)m2;
    const T w = (kz == 0 || 2 * kz == n) ? (T)1 : (T)2;
    const cplx<T> v = F[q];
    const T vr = v.x * invN, vi = v.y * invN;   // f~(G)
    const T a2 = vr * vr + vi * vi;
    cplx<T> o;
    if (fid == 0) {
      T orr = 0, oi = 0;
      if (g.hartree && m2 > 0) {
        const T c = fourpi / G2;
        acc[0].add(w * halfOm * c * a2);
        orr = c * vr; oi = c * vi;
      }
      if (with_loc) {                           // zero beyond the cutoff
        const cplx<T> vl = vbuf[q];
        acc[1].add(w * Om * (vr * vl.x + vi * vl.y));
        orr += vl.x; oi += vl.y;
      }
      o = mk<T>(orr, oi);
    } else if (fid == 1) {
      const T k = g.K[m2];
      acc[2].add(w * Om * k * a2);
      o = mk<T>(k * vr, k * vi);
    } else if (g.prec != nullptr) {
      // preconditioning pass: P f = IFFT[p(G) f~] (no energies)
      const T pg = g.prec[m2];
      o = mk<T>(pg * vr, pg * vi);
    } else {
      acc[3].add(w * halfOm * G2 * a2);
      if (sp.merged) {
        const T k = g.K[m2];
        acc[2].add(w * Om * k * a2);
        const T c = k + (T)0.5 * G2;
        o = mk<T>(c * vr, c * vi);
      } else {
        o = mk<T>(G2 * vr, G2 * vi);
      }
    }
    F[q] = o;
  }
  __syncthreads();
  cplx<T>* other = (F == buf0) ? buf1 : buf0;
  cplx<T>* res = fft_smem<T, +1>(F, other, pn, J, 1, J, tw_n);
  for (int q = threadIdx.x; q < n * J; q += blockDim.x) {
    const int kx = q >> lgJ, j = q & (J - 1);
    if (j < jn) base[(size_t)kx * plane + j] = res[q];
  }
  // the tile buffers are free now: reduce through them (dynamic smem is
  // sized to hold the tree scratch)
  const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
  block_sum_tree_raw<4, T>(acc, g.partials + b * 4, reinterpret_cast<typename TreeVal<T>::type*>(smem_raw));
}

// ---------------------------------------------------------------------------
// Final reduction of one evaluation, by the last block (fixed order:
// deterministic).  It only adds: out[0..3] = sums of the G-space columns
// (E_H, E_loc, E_NL, E_vW raw), out[4..11] = sums of the epilogue columns
// (F_TF, E_xc, int v_rest n, int g' d, int g'^2, int g' psi_t, int n,
// nonfinite count), all before the dV and scale factors.  The host, which
// reads them anyway, forms the energies, mu, the residual and the slope:
// GB300 issues FP64 at 1/64 of the FP32 rate, so even one thread's divisions
// and square roots here would be a serial tail of several microseconds.  For
// the same reason the partials are float-float pairs in FP32 plans and are
// added on the FP32 pipe.
template <typename T> struct FinArgs {
  using V = typename TreeVal<T>::type;
  const V* pg; int ng;          // G-space partials [ng][4]
  const V* pe; int ne;          // epilogue partials [ne][8]
  double* out;                  // [12]
};

template <typename T>
static __device__ void finalize_eval(const FinArgs<T>& f, typename TreeVal<T>::type* scr) {
  using V = typename TreeVal<T>::type;
  V acc[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) acc[q] = V{};
  const int nt = blockDim.x;
  // a thread's next rows' loads (32 values) are in flight together, added in
  // row order; this one block's pass over all partials is the kernel's tail
  for (int b0 = threadIdx.x; b0 < f.ng; b0 += 8 * nt) {
    V x[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int b = b0 + u * nt;
#pragma unroll
      for (int q = 0; q < 4; ++q) x[u][q] = b < f.ng ? __ldcg(f.pg + (size_t)b * 4 + q) : V{};
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = tree_add(acc[q], x[u][q]);
  }
  for (int b0 = threadIdx.x; b0 < f.ne; b0 += 4 * nt) {
    V x[4][8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int b = b0 + u * nt;
#pragma unroll
      for (int q = 0; q < 8; ++q) x[u][q] = b < f.ne ? __ldcg(f.pe + (size_t)b * 8 + q) : V{};
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[4 + q] = tree_add(acc[4 + q], x[u][q]);
  }
  const int pitch = nt + 1;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 12; ++q) scr[q * pitch + threadIdx.x] = acc[q];
  block_tree_core(12, scr);
  if (threadIdx.x < 12) f.out[threadIdx.x] = tree_get(scr[threadIdx.x * pitch]);
}

// ---------------------------------------------------------------------------
// 5. C2R along z + pointwise functional.
template <typename T> struct EpiArgs {
  int mode;              // 0: density given (write v); 1: psi + t d (write g');
                         // 3: preconditioning pass (write the psi field's real
                         // output to out; no functional, no sums)
  const T* rho;
  const T* psi;
  const T* d;
  T t, scale, alpha, T_e;   // converted on the host: no FP64 work in the kernels
  T cy;                  // pi^2 / (sqrt2 T^(3/2)): y = cy * n
  T mu_ref;              // g' is formed with v_rest - mu_ref (mode 1), see FinArgs
  int terms;             // OFDFT_TERM_* mask
  T* out;                // v (mode 0) or g' = psi_t v_rest + lap/2 (mode 1); may be null
  typename TreeVal<T>::type* partials;   // [gridDim.x][8], tree form (see GArgs)
  FinArgs<T> fin;        // final reduction, done by the last block to finish
  unsigned int* counter;
  // mode 3 only: with pyout non-null, also pyout = out - pold (the minimiser's
  // P y = P g_new - P g_old)
  const T* pold;
  T* pyout;
  const double* dsc;     // when set, scale = dsc[0] and t = dsc[2] (a trial formed on the device)
  int fd64;              // FP32 plans: invert the Fermi-Dirac integral in FP64 (y = cy_d n in FP64)
  double cy_d;           // pi^2 / (sqrt2 T^(3/2)) in FP64, for fd64
};

// The pointwise functional at one grid point, shared by the z-pass epilogue
// kernels: from the point's density (mode 0) or psi and d (mode 1) and the
// inverse transforms of the active fields there (Hartree + local potential,
// the n^a field, the psi field), the Thomas-Fermi and XC energy densities, the
// potential (mode 0) or g' (mode 1) written to out[at], and the block's
// partial sums acc: 0 F_TF, 1 E_xc, 2 int v_rest n, 3 int g' d, 4 int g'^2,
// 5 int g' psi_t, 6 int n, 7 nonfinite count.
template <typename T> struct EpiPoint {
  bool has_n, has_na, has_psi, merged;
  T Te, cy, alpha, nmin, tstep, tscale, muref;
  __device__ __forceinline__ EpiPoint(const Spectra<T>& sp, const EpiArgs<T>& a)
      : has_n(sp.s[0] != nullptr), has_na(sp.s[1] != nullptr), has_psi(sp.s[2] != nullptr),
        merged(sp.merged != 0), Te(a.T_e), cy(a.cy), alpha(a.alpha), nmin((T)kNmin),
        tstep(a.dsc ? (T)a.dsc[2] : a.t), tscale(a.dsc ? (T)a.dsc[0] : a.scale), muref(a.mu_ref) {}
  __device__ __forceinline__ void point(const EpiArgs<T>& a, T pv, T dq, T hv, T kv, T lv, size_t at,
                                        AccShort<T> (&acc)[8]) const {
    T psit, nval;
    if (a.mode == 0) {
      nval = pv;
      psit = sqrt(fmax(nval, (T)0));
    } else {
      psit = pv + tstep * dq;
      nval = tscale * psit * psit;
    }
    const T nf = fmax(nval, nmin);
    T vrest = 0;
    if (a.terms & 1) {              // TF
      if (sizeof(T) == 4 && a.fd64) {
        // FP64 inversion from the stored density value; f_TF formed in FP64
        double eta, p;
        fd_eta_p((double)nf * a.cy_d, eta, p);
        const double te = (double)Te;
        vrest += (T)(te * eta);
        acc[0].add((T)((double)nf * te * (eta - p)));
      } else {
        T eta, p;
        fd_eta_p(nf * cy, eta, p);
        vrest += Te * eta;
        acc[0].add(nf * Te * (eta - p));
      }
    }
    if (a.terms & 8) {              // XC
      T exc, vxc;
      pz81<T>(nf, exc, vxc);
      vrest += vxc;
      acc[1].add(nval * exc);
    }
    finish(a, psit, nval, nf, dq, vrest, hv, kv, lv, at, acc);
  }
  // the nonlocal and G-space contributions, the output and the sums
  __device__ __forceinline__ void finish(const EpiArgs<T>& a, T psit, T nval, T nf, T dq, T vrest, T hv, T kv,
                                         T lv, size_t at, AccShort<T> (&acc)[8]) const {
    if (has_n) vrest += hv;
    if (has_na) vrest += (T)2 * alpha * pow_t<T>(nf, alpha - (T)1) * kv;
    // psi field: -lap(psi), or W = IFFT[(K + G^2/2) psi~] when merged
    const T lw = has_psi ? lv : (T)0;
    const T extra = merged ? lw : (T)0.5 * lw;     // psi v_NL + (-lap psi)/2 when merged
    acc[2].add(vrest * nval);
    acc[6].add(nval);
    // g' = psi (v_rest - mu_ref) + lap/2: near convergence mu_ref is close to
    // mu, so the projection g = 2 scale (g' - (mu - mu_ref) psi) cancels little
    const T gp = psit * (vrest - muref) + extra;
    T* __restrict__ gout = a.out;
    if (a.mode == 0) {
      const T phi = fmax(psit, (T)kPhiMin);
      const T v = vrest + extra / phi;
      if (gout) gout[at] = v;
      // residual pieces with psi = sqrt(rho), scale 1: g' = psi v_rest + lap/2
      if (!isfinite(v)) acc[7].add((T)1);
    } else {
      if (gout) gout[at] = gp;
      acc[3].add(gp * dq);
      if (!isfinite(gp)) acc[7].add((T)1);
    }
    acc[4].add(gp * gp);
    acc[5].add(gp * psit);
  }
};

// smem: stg[nact][R][nh] (complex; field f's real rows overwrite its own
// staging once it has been pre-processed) | buf0[R][P] | buf1[R][P] |
// pin[2][R][n] (the block's rho, or psi and d, copied in with the spectra so
// that the pointwise loop does not wait on memory)
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_zinv_epi(Spectra<T> sp, EpiArgs<T> a, FftPlan1 ph,
                                                     const cplx<T>* __restrict__ tw_h,
                                                     const cplx<T>* __restrict__ tw_n, int n, int R, int P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int h = n / 2, nh = h + 1;
  cplx<T>* stg = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* buf0 = stg + (size_t)sp.nact * R * nh;
  cplx<T>* buf1 = buf0 + zbuf_elems(n, R, P);
  T* pin = reinterpret_cast<T*>(buf1 + zbuf_elems(n, R, P));
  const size_t row0 = (size_t)blockIdx.x * R;
  const int Rfull = R;
  R = (int)min((size_t)R, (size_t)n * n - row0);     // rows in this block
  const int tot = R * n;
  const size_t off = row0 * n;
  const unsigned Mh = qmagic(h), MR = qmagic(R);
  const size_t nn = (size_t)n * n;
  // all spectrum rows of the block in flight at once (tiled layout: contiguous
  // per field; plane layout: runs of R rows per kz)
  for (int f = 0; f < sp.nact; ++f) {
    cplx<T>* dst = stg + (size_t)f * Rfull * nh;
    if (sp.planes) {
      const cplx<T>* in = sp.s[sp.idx[f]] + row0;
      for (int q = threadIdx.x; q < R * nh; q += blockDim.x) {
        const int k = qdiv(q, R, MR), r = q - k * R;
        cp_async_c(dst + r * nh + k, in + (size_t)k * nn + r, true);
      }
    } else {
      const cplx<T>* in = sp.s[sp.idx[f]] + row0 * nh;
      for (int q = threadIdx.x; q < R * nh; q += blockDim.x) cp_async_c(dst + q, in + q, true);
    }
  }
  {
    // rows of rho (mode 0) or psi and d (mode 1) in 8-byte pieces: the block
    // starts on an 8-byte boundary (n even, or an even number of rows per
    // block); an odd element count leaves one element for a 4-byte copy
    constexpr int E = 8 / sizeof(T);
    const int pieces = tot / E;
    // (mode 3: the previous output pold, when P y = out - pold is wanted)
    const T* src0 = a.mode == 0 ? a.rho : (a.mode == 3 ? a.pold : a.psi);
    const bool want = a.mode != 3 || a.pyout != nullptr;
    const int npc = want ? pieces : 0;
    for (int q = threadIdx.x; q < npc; q += blockDim.x) {
      cp_async<8>(pin + q * E, src0 + off + q * E, true);
      if (a.mode == 1) cp_async<8>(pin + (size_t)Rfull * n + q * E, a.d + off + q * E, true);
    }
    if (want && pieces * E < tot && threadIdx.x == 0) {
      const int q = tot - 1;                 // E = 2 and tot odd: the last float
      cp_async<sizeof(T)>(pin + q, src0 + off + q, true);
      if (a.mode == 1) cp_async<sizeof(T)>(pin + (size_t)Rfull * n + q, a.d + off + q, true);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  // realf of field f = the first R*n reals of its staging slot
  T* realf[3];
  for (int f = 0; f < 3; ++f) realf[f] = nullptr;
  for (int f = 0; f < sp.nact; ++f) {
    const int fid = sp.idx[f];
    cplx<T>* in = stg + (size_t)f * Rfull * nh;
    if (n & 1) {
      // odd n: rows 2p and 2p + 1 from one length-n inverse transform of
      // Z[k] = A[k] + i B[k], A and B the rows' spectra extended by
      // A[n-k] = A*[k] (the imaginary parts at k = 0 dropped, as a real
      // inverse transform does); the result is a + i b
      const int npair = (R + 1) >> 1;
      const unsigned Mn = qmagic(n);
      for (int q = threadIdx.x; q < npair * n; q += blockDim.x) {
        const int pr = qdiv(q, n, Mn), k = q - pr * n;
        const int rb = 2 * pr + 1;
        const bool lo = k < nh;
        const int kk = lo ? k : n - k;
        cplx<T> A = in[2 * pr * nh + kk];
        cplx<T> B = rb < R ? in[rb * nh + kk] : mk<T>((T)0, (T)0);
        if (k == 0) { A.y = 0; B.y = 0; }
        if (!lo) { A.y = -A.y; B.y = -B.y; }
        buf0[pr * P + k] = mk<T>(A.x - B.y, A.y + B.x);
      }
      __syncthreads();                                 // staging slot f is now free
      cplx<T>* z = fft_smem<T, +1>(buf0, buf1, ph, 1, P, npair, tw_h);
      T* dst = reinterpret_cast<T*>(in);
      for (int q = threadIdx.x; q < tot; q += blockDim.x) {
        const int r = qdiv(q, n, Mn), j = q - r * n;
        const cplx<T> v = z[(r >> 1) * P + j];
        dst[q] = (r & 1) ? v.y : v.x;
      }
      realf[fid] = dst;
      __syncthreads();
      continue;
    }
    // Z[k] = (X[k] + X*[h-k]) + i W^-k (X[k] - X*[h-k]),  k = 0..h-1
    for (int q = threadIdx.x; q < R * h; q += blockDim.x) {
      const int r = qdiv(q, h, Mh), k = q - r * h;
      const cplx<T> xk = in[r * nh + k];
      const cplx<T> xc = cconj(in[r * nh + (h - k)]);
      const cplx<T> e = cadd(xk, xc);
      const cplx<T> o = cmul(cconj(tw_n[k]), csub(xk, xc));
      buf0[r * P + k] = mk<T>(e.x - o.y, e.y + o.x);   // e + i o
    }
    __syncthreads();                                   // staging slot f is now free
    cplx<T>* z = fft_smem<T, +1>(buf0, buf1, ph, 1, P, R, tw_h);
    // real pairs land as one 8- or 16-byte store (R h complex <= R nh slots)
    cplx<T>* dst = in;
    for (int q = threadIdx.x; q < R * h; q += blockDim.x) {
      const int r = qdiv(q, h, Mh), k = q - r * h;
      dst[r * h + k] = z[r * P + k];
    }
    realf[fid] = reinterpret_cast<T*>(in);
    __syncthreads();
  }
  // pointwise functional
  if (a.mode == 3) {
    // every block takes this branch: no partial sums, no final reduction
    const T* fP = realf[2];
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
      const T v = fP[q];
      a.out[off + q] = v;
      if (a.pyout) a.pyout[off + q] = v - pin[q];
    }
    return;
  }
  const T* fH = realf[0];
  const T* fK = realf[1];
  const T* fL = realf[2];
  const EpiPoint<T> ep(sp, a);
  AccShort<T> acc[8];
  const T* pd = pin + (size_t)Rfull * n;
  for (int q = threadIdx.x; q < tot; q += blockDim.x)
    ep.point(a, pin[q], a.mode != 0 ? pd[q] : (T)0, fH ? fH[q] : (T)0, fK ? fK[q] : (T)0, fL ? fL[q] : (T)0,
             off + q, acc);
  typename TreeVal<T>::type* scr = reinterpret_cast<typename TreeVal<T>::type*>(smem_raw);
  block_sum_tree_raw<8, T>(acc, a.partials + (size_t)blockIdx.x * 8, scr);
  if (arrive_last(a.counter)) {
    finalize_eval<T>(a.fin, scr);
    if (threadIdx.x == 0) *a.counter = 0u;
  }
}

}  // namespace ofdft
