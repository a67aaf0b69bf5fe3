// Per-cell setup kernels: ion structure factor and local pseudopotential,
// Ewald ion-ion energy, the nonlocal kernel table K(|G|), S_ei shell sums.
#pragma once
#include "common.cuh"
#include "passes.cuh"

namespace ofdft {

// ---------------------------------------------------------------------------
// Structure factor on the half spectrum.  Phases factorise per axis:
// exp(-i G.R) = e_x(m_x) e_y(m_y) e_z(m_z) with e_d(m) = exp(-2 pi i m R_d / L);
// ph[(I*3 + d)*n + k] holds them (FP64, k in FFT order).
static __global__ void k_phases(const double* __restrict__ pos, int n_ion, int n, double L,
                         double2* __restrict__ ph) {
  const int tot = n_ion * 3 * n;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += gridDim.x * blockDim.x) {
    const int k = q % n, d = (q / n) % 3, I = q / (3 * n);
    const int m = k <= (n - 1) / 2 ? k : k - n;
    double f = pos[I * 3 + d] / L;
    f -= floor(f);                       // wrap into [0, 1)
    // angle = -2 pi m f; reduce m f modulo 1 before the trig call
    double mf = (double)m * f;
    mf -= rint(mf);
    double s, c;
    sincospi(-2.0 * mf, &s, &c);
    ph[q] = make_double2(c, s);
  }
}

// S(G) = sum_I exp(-i G.R_I) and S_Z(G) = sum_I Z_I exp(-i G.R_I) on the half
// spectrum; V_loc(G) = (1/Omega) v~(G) S_Z(G) with the common smoothing radius
// rc; the Ewald reciprocal sum (2 pi / Omega) sum_{G != 0} exp(-G^2/4eta^2)/G^2
// |S_Z|^2 accumulated on the way.  A block takes kStructRows (kx, ky) rows, one
// per warp, lanes over kz; the ions go in chunks of ch, whose kz phases are
// staged in shared memory once for all rows of the block (with the rows' (kx,
// ky) phase products).  Rows whose smallest |G|^2 exceeds g2max are written as
// zero (their V_loc and Ewald weights are below double precision) unless
// full != 0.
//   sf_tab[m^2] = (v~(G)/Omega per unit charge, (2 pi/Omega) exp(-G^2/(4 eta^2))/G^2),
// the second 0 at m^2 = 0: both depend on |G| only and are tabulated once per
// plan in FP64, so no exponential is evaluated here.
// S_Z itself is kept as well (SZ_out), for the forces.
// Shared memory: ez[ch][nh] | xy[kStructRows][ch] (complex) | zz[ch] (T).
constexpr int kStructRows = 8;
constexpr int kStructMaxKJ = 9;     // kz per lane: nh <= 32 * 9

// UNI: every ion has the charge Z[0]; S_Z is then Z[0] S and is not summed.
template <typename T, bool UNI>
__global__ void __launch_bounds__(32 * kStructRows) k_struct(const double2* __restrict__ ph,
                                                             const double* __restrict__ Z, int n_ion, int n,
                                                             double L, const double2* __restrict__ sf_tab,
                                                             double g2max, int full, int mlim, int ch,
                                                             cplx<T>* __restrict__ S_out,
                                                             cplx<T>* __restrict__ vloc,
                                                             cplx<T>* __restrict__ SZ_out,
                                                             double* __restrict__ ew_partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int nh = n / 2 + 1;
  cplx<T>* ez = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* sxy = ez + (size_t)ch * nh;
  T* szz = reinterpret_cast<T*>(sxy + (size_t)kStructRows * ch);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // mlim < 0: every (kx, ky) row of the grid; mlim >= 0: the rows with |mx|,
  // |my| <= mlim (the caller has zeroed the other rows)
  const int side = 2 * mlim + 1;
  const int nrows = mlim < 0 ? n * n : side * side;
  auto row_of = [&](int rw, int& kx, int& ky, int& mx, int& my) {
    if (mlim < 0) {
      kx = rw / n; ky = rw % n;
      mx = kx <= (n - 1) / 2 ? kx : kx - n;
      my = ky <= (n - 1) / 2 ? ky : ky - n;
    } else {
      mx = rw / side - mlim; my = rw % side - mlim;
      kx = mx < 0 ? mx + n : mx; ky = my < 0 ? my + n : my;
    }
  };
  const int row = blockIdx.x * kStructRows + warp;
  int kx = 0, ky = 0, mx = 0, my = 0;
  const bool valid = row < nrows;
  if (valid) row_of(row, kx, ky, mx, my);
  const double tp = 2.0 * kPi / L;
  const bool skip = !full && tp * tp * (double)(mx * mx + my * my) > g2max;
  T sr[kStructMaxKJ], si[kStructMaxKJ], zr[kStructMaxKJ], zi[kStructMaxKJ];
#pragma unroll
  for (int j = 0; j < kStructMaxKJ; ++j) { sr[j] = 0; si[j] = 0; zr[j] = 0; zi[j] = 0; }
  for (int I0 = 0; I0 < n_ion; I0 += ch) {
    const int cnt = min(ch, n_ion - I0);
    __syncthreads();
    for (int q = threadIdx.x; q < cnt * nh; q += blockDim.x) {
      const int c = q / nh, kz = q - c * nh;
      const double2 e = ph[((size_t)(I0 + c) * 3 + 2) * n + kz];
      ez[q] = mk<T>((T)e.x, (T)e.y);
    }
    for (int q = threadIdx.x; q < kStructRows * cnt; q += blockDim.x) {
      const int r = q / cnt, c = q - r * cnt;
      const int rw = blockIdx.x * kStructRows + r;
      cplx<T> v = mk<T>((T)0, (T)0);
      if (rw < nrows) {
        int qx, qy, px, py;
        row_of(rw, qx, qy, px, py);
        const double2 ex = ph[((size_t)(I0 + c) * 3 + 0) * n + qx];
        const double2 ey = ph[((size_t)(I0 + c) * 3 + 1) * n + qy];
        v = mk<T>((T)(ex.x * ey.x - ex.y * ey.y), (T)(ex.x * ey.y + ex.y * ey.x));
      }
      sxy[r * ch + c] = v;
    }
    for (int c = threadIdx.x; c < cnt; c += blockDim.x) szz[c] = (T)Z[I0 + c];
    __syncthreads();
    if (valid && !skip) {
      for (int c = 0; c < cnt; ++c) {
        const cplx<T> xy = sxy[warp * ch + c];
        const T zc = szz[c];
        const cplx<T>* e = ez + (size_t)c * nh;
#pragma unroll
        for (int j = 0; j < kStructMaxKJ; ++j) {
          const int kz = lane + 32 * j;
          if (kz < nh) {
            const cplx<T> w = e[kz];
            const T pr = xy.x * w.x - xy.y * w.y, pi = xy.x * w.y + xy.y * w.x;
            sr[j] += pr; si[j] += pi;
            if constexpr (!UNI) { zr[j] += zc * pr; zi[j] += zc * pi; }
          }
        }
      }
    }
  }
  if constexpr (UNI) {
    const T z0 = (T)Z[0];
#pragma unroll
    for (int j = 0; j < kStructMaxKJ; ++j) { zr[j] = z0 * sr[j]; zi[j] = z0 * si[j]; }
  }
  double ew = 0;
  if (valid) {
    const size_t rowoff = ((size_t)kx * n + ky) * nh;
#pragma unroll
    for (int j = 0; j < kStructMaxKJ; ++j) {
      const int kz = lane + 32 * j;
      if (kz >= nh) continue;
      if (skip) {
        if (S_out) S_out[rowoff + kz] = mk<T>(0, 0);
        vloc[rowoff + kz] = mk<T>(0, 0);
        SZ_out[rowoff + kz] = mk<T>(0, 0);
        continue;
      }
      const int m2 = mx * mx + my * my + kz * kz;
      if (S_out) S_out[rowoff + kz] = mk<T>(sr[j], si[j]);
      SZ_out[rowoff + kz] = mk<T>(zr[j], zi[j]);
      const double2 f = sf_tab[m2];
      vloc[rowoff + kz] = mk<T>((T)(f.x * (double)zr[j]), (T)(f.x * (double)zi[j]));
      const double w = (kz == 0 || 2 * kz == n) ? 1.0 : 2.0;
      ew += w * f.y * ((double)zr[j] * (double)zr[j] + (double)zi[j] * (double)zi[j]);
    }
  }
  double v[1] = {ew}, out[1];
  block_sum<1>(v, red, out);
  if (threadIdx.x == 0) ew_partial[blockIdx.x] = out[0];
}

// ---------------------------------------------------------------------------
// Ewald: real-space pair sum (all pairs I, J and lattice images within rcut).
// Each pair's displacement is taken at minimum image (|d| <= L/2 per axis), so
// images a with |a| <= nimg = ceil(rcut/L + 1/2) per axis cover every
// distance below rcut.  A block walks its share of the (pair, image)
// combinations 256 at a time, compacts the ones inside rcut into shared
// memory (warp ballots and a block prefix, in combination order) and only
// then evaluates erfc, on dense warps: the FP64 erfc is by far the costliest
// step, and fewer than 1% of the combinations are inside.  Fixed order
// throughout, so the sum is deterministic.
static __global__ void __launch_bounds__(256) k_ewald_real(const double* __restrict__ pos,
                                                           const double* __restrict__ Z, int n_ion, double L,
                                                           double eta, double rcut, int nimg,
                                                           double* __restrict__ partial) {
  __shared__ double red[32];
  __shared__ double sr[256], sz[256];
  __shared__ int wcount[8], wbase[8], total;
  const int side = 2 * nimg + 1;
  const long nim3 = (long)side * side * side;
  const long tot = (long)n_ion * n_ion * nim3;
  const long per = (tot + gridDim.x - 1) / gridDim.x;
  const long q0 = (long)blockIdx.x * per, q1 = min(tot, q0 + per);
  const double rc2 = rcut * rcut;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double acc = 0;
  for (long base = q0; base < q1; base += blockDim.x) {
    const long q = base + threadIdx.x;
    bool inside = false;
    double r = 0, zz = 0;
    if (q < q1) {
      const long p = q / nim3;
      const int im = (int)(q - p * nim3);
      const int I = (int)(p / n_ion), J = (int)(p % n_ion);
      const int a = im / (side * side) - nimg, b = (im / side) % side - nimg, c = im % side - nimg;
      double x = pos[I * 3] - pos[J * 3], y = pos[I * 3 + 1] - pos[J * 3 + 1], z = pos[I * 3 + 2] - pos[J * 3 + 2];
      const double iL = 1.0 / L;     // uniform: folded to one reciprocal per thread
      x -= L * rint(x * iL); y -= L * rint(y * iL); z -= L * rint(z * iL);
      x += a * L; y += b * L; z += c * L;
      const double r2 = x * x + y * y + z * z;
      inside = r2 > 1e-24 && r2 < rc2;
      if (inside) { r = sqrt(r2); zz = Z[I] * Z[J]; }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, inside);
    if (lane == 0) wcount[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { wbase[w] = s; s += wcount[w]; }
      total = s;
    }
    __syncthreads();
    if (inside) {
      const int slot = wbase[wid] + __popc(bal & ((1u << lane) - 1u));
      sr[slot] = r; sz[slot] = zz;
    }
    __syncthreads();
    if ((int)threadIdx.x < total) acc += 0.5 * sz[threadIdx.x] * erfc(eta * sr[threadIdx.x]) / sr[threadIdx.x];
    __syncthreads();
  }
  double v[1] = {acc}, out[1];
  block_sum<1>(v, red, out);
  if (threadIdx.x == 0) partial[blockIdx.x] = out[0];
}

// ---------------------------------------------------------------------------
// Nonlocal kernel table.  One thread per integer m^2 in [0, nm2).
//   chi0(q;T) = -1/(pi^2 q) int_0^kmax k f(k) ln|(2k+q)/(2k-q)| dk
// with f(k) = 1/(1 + exp((k^2/2 - mu0)/T)).  The 4k/q part of the logarithm
// integrates to 4 pi^2 nbar / q exactly, so only the excess over it is
// integrated (no cancellation when -1/chi0 is compared with q^2/(4 nbar)).
// On the panel holding the logarithmic singularity c = q/2 the integrand is
// written with g(k) = k f(k) as g [ln(2k+q) - 4k/q] - (g - g(c)) ln|2k-q| plus
// g(c) int ln|2k-q| in closed form, and graded geometrically toward c; panel
// widths stay below pi T / k_F so the Fermi edge is resolved.
//   K(q) = [-1/chi0 - dmu0/dn - q^2/(4 nbar)] / (2 a^2 nbar^(2a-2)),  K(0) = 0.
struct KernArgs {
  double L, nbar, T, mu0, dmudn, alpha;
  int nm2;
};

static __device__ __forceinline__ double occ_fd(double k, double mu0, double T) {
  const double u = (0.5 * k * k - mu0) / T;
  if (u > 0) { const double e = exp(-u); return e / (1.0 + e); }
  return 1.0 / (1.0 + exp(u));
}

// 10-point Gauss-Legendre on [-1, 1]
static __device__ __constant__ double c_glx[10] = {
    -0.97390652851717172008, -0.86506336668898451073, -0.67940956829902440623, -0.43339539412924719080,
    -0.14887433898163121088, 0.14887433898163121088, 0.43339539412924719080, 0.67940956829902440623,
    0.86506336668898451073, 0.97390652851717172008};
static __device__ __constant__ double c_glw[10] = {
    0.06667134430868813759, 0.14945134915058059315, 0.21908636251598204400, 0.26926671930999635509,
    0.29552422172787993740, 0.29552422172787993740, 0.26926671930999635509, 0.21908636251598204400,
    0.14945134915058059315, 0.06667134430868813759};

// Gauss-Legendre on [a, b] of g(k) [ln|(2k+q)/(2k-q)| - 4k/q], for panels that
// do not contain q/2: x = 2k/q, 2 (atanh x - x) below 1, ln((x+1)/(x-1)) - 2x above.
static __device__ double lind_panel_plain(double a, double b, double q, double mu0, double T) {
  const double h = 0.5 * (b - a), m = 0.5 * (b + a);
  double s = 0;
#pragma unroll
  for (int j = 0; j < 10; ++j) {
    const double k = m + h * c_glx[j];
    const double x = 2.0 * k / q;
    const double e = x < 1.0 ? 2.0 * (atanh(x) - x) : log((x + 1.0) / (x - 1.0)) - 2.0 * x;
    s += c_glw[j] * k * occ_fd(k, mu0, T) * e;
  }
  return s * h;
}

// Same integrand near q/2, written g [ln(2k+q) - 4k/q] - (g - g(c)) ln|2k - q|
// (the g(c) ln|2k - q| part is added in closed form by the caller).
static __device__ double lind_panel_split(double a, double b, double q, double c, double gc, double mu0,
                                          double T) {
  const double h = 0.5 * (b - a), m = 0.5 * (b + a);
  double s = 0;
#pragma unroll
  for (int j = 0; j < 10; ++j) {
    const double k = m + h * c_glx[j];
    const double g = k * occ_fd(k, mu0, T);
    const double d = fabs(2.0 * k - q);
    double v = g * (log(2.0 * k + q) - 4.0 * k / q);
    if (d > 0) v -= (g - gc) * log(d);
    s += c_glw[j] * v;
  }
  return s * h;
}

// One warp per m^2 (kKernWarps warps per block): the lanes take the plain
// panels and the graded levels in turn, and the lane sums are added by a
// fixed shuffle tree, so the result does not depend on the launch.  (One
// thread per m^2 left a small grid's table to a few hundred threads, each
// integrating thousands of panels: 5.6 ms at 16^3.)
constexpr int kKernWarps = 4;
static __global__ void __launch_bounds__(32 * kKernWarps) k_kernel_table(KernArgs a, double* __restrict__ Kout) {
  const int lane = threadIdx.x & 31;
  const int m2 = blockIdx.x * kKernWarps + (threadIdx.x >> 5);
  if (m2 >= a.nm2) return;                            // whole warps leave together
  if (m2 == 0) { if (lane == 0) Kout[0] = 0.0; return; }
  const double q = 2.0 * kPi / a.L * sqrt((double)m2);
  const double T = a.T, mu0 = a.mu0;
  const double kmax = sqrt(2.0 * fmax(mu0 + 45.0 * T, 45.0 * T));
  const double kedge = mu0 > 0 ? sqrt(2.0 * mu0) : sqrt(2.0 * T);
  double hmax = fmin(kmax / 16.0, 0.5 * kPi * T / fmax(kedge, sqrt(2.0 * T)));
  const int npan = min(4096, (int)ceil(kmax / hmax));
  const double h = kmax / npan;     // plain panel width
  const double c = 0.5 * q;
  const double gc = c * occ_fd(c, mu0, T);
  // closed form of int ln|2k - q| dk: (1/2) [u ln|u| - u], u = 2k - q
  auto F = [](double u) { return u == 0 ? 0.0 : u * log(fabs(u)) - u; };
  double part = 0;   // this lane's share of int_0^kmax k f(k) [ln|(2k+q)/(2k-q)| - 4k/q] dk
  // graded region [ga, gb] around c (at least 2 panel widths on each side, so
  // that every plain panel stays >= 2h away from the singularity)
  const bool sing = c < kmax + 2.0 * h;
  const double ga = sing ? fmax(0.0, c - 2.0 * h) : kmax;
  const double gb = sing ? fmin(kmax, c + 2.0 * h) : kmax;
  // plain panels on [0, ga] and [gb, kmax]
  auto plain = [&](double a0, double b0) {
    if (b0 <= a0) return;
    const int np = max(1, (int)ceil((b0 - a0) / h));
    const double hh = (b0 - a0) / np;
    for (int p = lane; p < np; p += 32) part += lind_panel_plain(a0 + p * hh, a0 + (p + 1) * hh, q, mu0, T);
  };
  plain(0.0, ga);
  plain(gb, kmax);
  if (sing && gb > ga) {
    // split at c (if inside), grade geometrically toward c from both ends:
    // level l covers [cl - w 2^-l, cl - w 2^-(l+1)] on the left (w = cl - ga)
    // and [cl + w' 2^-(l+1), cl + w' 2^-l] on the right (w' = gb - cl), down
    // to widths of 1e-15 (c + h), at most 48 levels a side
    const double cl = fmin(fmax(c, ga), gb);
    const double wl = cl - ga, wr = gb - cl, wmin = 1e-15 * (c + h);
    for (int lev = lane; lev < 96; lev += 32) {
      const bool left = lev < 48;
      const int l = left ? lev : lev - 48;
      const double w = (left ? wl : wr) * ldexp(1.0, -l);
      if (!(w > wmin)) continue;
      if (left) part += lind_panel_split(cl - w, cl - 0.5 * w, q, c, gc, mu0, T);
      else part += lind_panel_split(cl + 0.5 * w, cl + w, q, c, gc, mu0, T);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane != 0) return;
  double integral = part;
  if (sing && gb > ga) integral -= gc * 0.5 * (F(2.0 * gb - q) - F(2.0 * ga - q));
  // chi0 = -(4 nbar / q^2)(1 + eps);  -1/chi0 - q^2/(4 nbar) = -(q^2/(4 nbar)) eps / (1 + eps)
  const double eps = integral * q / (4.0 * kPi * kPi * a.nbar);
  const double resp_excess = -q * q / (4.0 * a.nbar) * eps / (1.0 + eps);
  const double denom = 2.0 * a.alpha * a.alpha * pow(a.nbar, 2.0 * a.alpha - 2.0);
  Kout[m2] = (resp_excess - a.dmudn) / denom;
}

// Launch shape of k_kernel_table for nm2 entries.
inline int kernel_table_blocks(int nm2) { return (nm2 + kKernWarps - 1) / kKernWarps; }

// I_{-1/2}(eta) = int_0^inf 2 / (1 + exp(t^2 - eta)) dt at the mean density,
// FP64: 400 panels of 10-point Gauss-Legendre, one panel per thread (one
// block of kMeanThreads), summed by a fixed tree.
constexpr int kMeanThreads = 512;
static __global__ void __launch_bounds__(kMeanThreads) k_mean_density(double y, double T, double* out) {
  __shared__ double red[kMeanThreads];
  double eta, p;
  fd_eta_p(y, eta, p);
  const double tmax = sqrt(fmax(eta, 0.0) + 60.0);
  const int npan = 400;
  const double h = tmax / npan;
  double s = 0;
  for (int i = threadIdx.x; i < npan; i += blockDim.x) {
    const double a = i * h, m = a + 0.5 * h;
    for (int j = 0; j < 10; ++j) {
      const double t = m + 0.5 * h * c_glx[j];
      const double u = t * t - eta;
      const double f = u > 0 ? exp(-u) / (1.0 + exp(-u)) : 1.0 / (1.0 + exp(u));
      s += c_glw[j] * 2.0 * f;
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double im = red[0] * 0.5 * h;
  out[0] = eta;
  out[1] = T * eta;                                                      // mu0
  out[2] = 2.0 * kPi * kPi / (1.4142135623730950488 * sqrt(T) * im);     // dmu0/dn
  out[3] = im;
}

// ---------------------------------------------------------------------------
// Structure-factor shells: block s sums over the half-spectrum entries of
// shell s (CSR lists built on the host; w = Hermitian weight), FP64, fixed
// order.  out[3 s] = sum w Re[n~ S*] scale, out[3 s + 1] = sum w |S|^2,
// out[3 s + 2] = sum w.
template <typename T>
__global__ void __launch_bounds__(256) k_sei_shells(const cplx<T>* __restrict__ nt, const cplx<T>* __restrict__ S,
                                                    const int* __restrict__ ptr, const long long* __restrict__ idx,
                                                    const float* __restrict__ wgt, double scale,
                                                    double* __restrict__ out) {
  __shared__ double red[3 * 32];
  const int s = blockIdx.x;
  double acc[3] = {0, 0, 0};
  for (int e = ptr[s] + threadIdx.x; e < ptr[s + 1]; e += blockDim.x) {
    const long long q = idx[e];
    const cplx<T> a = nt[q], b = S[q];
    const double w = (double)wgt[e];
    acc[0] += w * ((double)a.x * (double)b.x + (double)a.y * (double)b.y) * scale;
    acc[1] += w * ((double)b.x * (double)b.x + (double)b.y * (double)b.y);
    acc[2] += w;
  }
  double o[3];
  block_sum<3>(acc, red, o);
  if (threadIdx.x == 0) { out[3 * s] = o[0]; out[3 * s + 1] = o[1]; out[3 * s + 2] = o[2]; }
}

// out[c] = sum_r partial[r * cols + c] in a fixed order; one block, cols <= blockDim.x
static __global__ void k_sum_columns(const double* __restrict__ partial, int rows, int cols, double* __restrict__ out) {
  block_sum_columns(partial, rows, cols, out, nullptr);
}

}  // namespace ofdft

namespace ofdft {

// ---------------------------------------------------------------------------
// Hellmann-Feynman forces at a given density (same derivation as the energy:
// at fixed n the ions enter only through E_loc and the Ewald energy).
//   F_I = -Z_I sum_G Im[qq(G) e_I(G)] G  +  Ewald real-space part,
//   e_I(G) = exp(-i G.R_I),  qq(G) = w(G) conj(vfac(G) n~(G) + efac(G) A(G)),
//   A(G) = sum_J Z_J exp(-i G.R_J),  vfac = -4 pi exp(-G^2 rc^2/4)/G^2 (per unit Z),
//   efac = (4 pi / Omega) exp(-G^2/(4 eta^2))/G^2,
// over the listed G (0 < |G|^2 within the local and Ewald cutoffs, half
// spectrum with Hermitian weight w = 2, or 1 on the kz = 0 and n/2 planes).
// The G list and the signed m of each index are those of k_struct, so the
// forces are the exact derivative of the energy the evaluation computes.

// one thread per listed G: qq(G) = w conj(vfac n~ + efac S_Z), with S_Z(G) as
// k_struct formed it (plan precision)
template <typename T>
__global__ void k_forces_q(const cplx<T>* __restrict__ nt, const int4* __restrict__ gl,
                           const double2* __restrict__ gf, int ng, const cplx<T>* __restrict__ SZ, int n,
                           double invN, cplx<T>* __restrict__ qq) {
  const int nh = n / 2 + 1;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
    const int4 e = gl[g];
    const size_t q = ((size_t)e.x * n + e.y) * nh + e.z;
    const cplx<T> v = nt[q], A = SZ[q];
    const double2 f = gf[g];                        // (vfac, efac)
    const double w = (double)e.w;
    const double qr = f.x * (double)v.x * invN + f.y * (double)A.x;
    const double qi = f.x * (double)v.y * invN + f.y * (double)A.y;
    qq[g] = mk<T>((T)(w * qr), (T)(-w * qi));       // w conj(Q)
  }
}

// e_I phases in the plan's precision: pt[(I*3 + d)*n + k] = ph[...]
template <typename T>
__global__ void k_phases_t(const double2* __restrict__ ph, cplx<T>* __restrict__ pt, int tot) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += gridDim.x * blockDim.x)
    pt[q] = mk<T>((T)ph[q].x, (T)ph[q].y);
}

// one block per ion: F_I(G part) = -Z_I tp sum_G Im[qq e_I] m(G) -> out[I*3 .. I*3+2]
template <typename T>
__global__ void __launch_bounds__(256) k_forces_g(const cplx<T>* __restrict__ qq, const int4* __restrict__ gl,
                                                  int ng, const cplx<T>* __restrict__ pt,
                                                  const double* __restrict__ Z, int n, double tp,
                                                  double* __restrict__ out) {
  __shared__ typename TreeVal<T>::type scr[3 * 257];
  const int I = blockIdx.x;
  const cplx<T>* px = pt + (size_t)I * 3 * n;
  const cplx<T>* py = px + n;
  const cplx<T>* pz = py + n;
  Acc<T> acc[3];
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    const int4 e = gl[g];
    const cplx<T> a = px[e.x], b = py[e.y], c = pz[e.z];
    const cplx<T> ab = cmul(a, b);
    const cplx<T> eI = cmul(ab, c);
    const cplx<T> q = qq[g];
    const T im = q.x * eI.y + q.y * eI.x;          // Im[q e_I]
    const int mx = e.x <= (n - 1) / 2 ? e.x : e.x - n;
    const int my = e.y <= (n - 1) / 2 ? e.y : e.y - n;
    const int mz = e.z <= (n - 1) / 2 ? e.z : e.z - n;   // the phase tables' convention
    acc[0].add(im * (T)mx); acc[1].add(im * (T)my); acc[2].add(im * (T)mz);
  }
  double s[3];
  block_sum_tree<3, T>(acc, 3, s, scr);
  if (threadIdx.x < 3) out[(size_t)I * 3 + threadIdx.x] = -Z[I] * tp * s[threadIdx.x];
}

// Ewald real-space force on ion I = blockIdx.x / nsplit from the share
// blockIdx.x % nsplit of its (J, image) terms, FP64, into part[blockIdx.x * 3
// ..] (k_sum_force_parts adds the shares to the forces in a fixed order).  As
// in k_ewald_real, displacements are taken at minimum image (|a| <= nimg
// images per axis then cover every distance below rcut) and the in-range terms
// are compacted before their erfc and exp are evaluated.
static __global__ void __launch_bounds__(256) k_ewald_force_real(const double* __restrict__ pos,
                                                                 const double* __restrict__ Z, int n_ion, double L,
                                                                 double eta, double rcut, int nimg, int nsplit,
                                                                 double* __restrict__ part) {
  __shared__ double red[3 * 32];
  __shared__ double sx[256], sy[256], sz[256], sq[256];
  __shared__ int wcount[8], wbase[8], total;
  const int I = blockIdx.x / nsplit, sh = blockIdx.x % nsplit;
  const int side = 2 * nimg + 1;
  const int nim3 = side * side * side;
  const long tot = (long)n_ion * nim3;
  const long per = (tot + nsplit - 1) / nsplit;
  const long q0 = (long)sh * per, q1 = min(tot, q0 + per);
  const double rc2 = rcut * rcut;
  const double c2 = 2.0 * eta / 1.7724538509055160273;   // 2 eta / sqrt(pi)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double iL = 1.0 / L;
  double f[3] = {0, 0, 0};
  for (long base = q0; base < q1; base += blockDim.x) {
    const long q = base + threadIdx.x;
    bool inside = false;
    double x = 0, y = 0, z = 0, r2 = 0;
    if (q < q1) {
      const int J = (int)(q / nim3), im = (int)(q % nim3);
      const int a = im / (side * side) - nimg, b = (im / side) % side - nimg, c = im % side - nimg;
      x = pos[I * 3] - pos[J * 3]; y = pos[I * 3 + 1] - pos[J * 3 + 1]; z = pos[I * 3 + 2] - pos[J * 3 + 2];
      x -= L * rint(x * iL); y -= L * rint(y * iL); z -= L * rint(z * iL);
      x += a * L; y += b * L; z += c * L;
      r2 = x * x + y * y + z * z;
      inside = r2 > 1e-24 && r2 < rc2;
      if (inside) r2 = Z[I] * Z[J];     // reused below as the charge product
    }
    const unsigned bal = __ballot_sync(0xffffffffu, inside);
    if (lane == 0) wcount[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { wbase[w] = s; s += wcount[w]; }
      total = s;
    }
    __syncthreads();
    if (inside) {
      const int slot = wbase[wid] + __popc(bal & ((1u << lane) - 1u));
      sx[slot] = x; sy[slot] = y; sz[slot] = z; sq[slot] = r2;
    }
    __syncthreads();
    if ((int)threadIdx.x < total) {
      const double dx = sx[threadIdx.x], dy = sy[threadIdx.x], dz = sz[threadIdx.x];
      const double rr = dx * dx + dy * dy + dz * dz, r = sqrt(rr);
      const double s = sq[threadIdx.x] * (erfc(eta * r) / rr + c2 * exp(-eta * eta * rr) / r) / r;
      f[0] += s * dx; f[1] += s * dy; f[2] += s * dz;
    }
    __syncthreads();
  }
  double o[3];
  block_sum<3>(f, red, o);
  if (threadIdx.x == 0) {
    part[(size_t)blockIdx.x * 3 + 0] = o[0]; part[(size_t)blockIdx.x * 3 + 1] = o[1];
    part[(size_t)blockIdx.x * 3 + 2] = o[2];
  }
}

// out[I * 3 + d] += sum_s part[(I nsplit + s) * 3 + d], s in order; one thread per (I, d)
static __global__ void k_sum_force_parts(const double* __restrict__ part, int n_ion, int nsplit,
                                         double* __restrict__ out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_ion * 3; t += gridDim.x * blockDim.x) {
    const int I = t / 3, d = t - I * 3;
    double s = 0;
    for (int k = 0; k < nsplit; ++k) s += part[((size_t)I * nsplit + k) * 3 + d];
    out[t] += s;
  }
}

}  // namespace ofdft

namespace ofdft {

// ---------------------------------------------------------------------------
// Pressure P = -dF/dOmega under a homogeneous dilation (L, R_I -> lambda L,
// lambda R_I; n -> n / lambda^3; fixed T).  The local functionals contribute
// (1/Omega) int (n v - f): for TF that is n T p(y), for LDA xc n (v_xc - e_xc).
// partial[block][2] = (sum n T p, sum n (v_xc - e_xc)) over the grid.
template <typename T>
__global__ void __launch_bounds__(256) k_pressure_r(const T* __restrict__ rho, size_t N, T cy, T Te, int terms,
                                                    double* __restrict__ partial, int fd64, double cy_d) {
  __shared__ typename TreeVal<T>::type scr[2 * 257];
  Acc<T> acc[2];
  const T nmin = (T)kNmin;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    const T nval = rho[q];
    const T nf = fmax(nval, nmin);
    if (terms & 1) {
      if (sizeof(T) == 4 && fd64) {          // FP64 inversion, as in the evaluation
        double eta, p;
        fd_eta_p((double)nf * cy_d, eta, p);
        acc[0].add((T)((double)nf * (double)Te * p));
      } else {
        T eta, p;
        fd_eta_p(nf * cy, eta, p);
        acc[0].add(nf * Te * p);
      }
    }
    if (terms & 8) {
      T exc, vxc;
      pz81<T>(nf, exc, vxc);
      acc[1].add(nval * (vxc - exc));
    }
  }
  block_sum_tree<2, T>(acc, 2, partial + (size_t)blockIdx.x * 2, scr);
}

// G-space parts over the half spectrum (tiled layout, Hermitian weight w):
//   partial[block][0] = sum w Re[n~* V_loc] c(G),  c = 3 at G = 0, 1 - G^2 rc^2/2 else
//                       (entries with |G|^2 <= g2cut, as in the energy),
//   partial[block][1] = sum w |(n^a)~|^2 pnl(m^2),  pnl = (3 - 6a) K + dK/dlambda.
// nt, wt are unnormalised transforms (times invN).  FP64 sums.
template <typename T>
__global__ void __launch_bounds__(256) k_pressure_g(const cplx<T>* __restrict__ nt, const cplx<T>* __restrict__ wt,
                                                    const cplx<T>* __restrict__ vloc, const double* __restrict__ pnl,
                                                    int n, double tp2, double g2cut, double rc2, double invN,
                                                    double* __restrict__ partial) {
  __shared__ double red[2 * 32];
  const int nh = n / 2 + 1;
  const size_t NH = (size_t)n * n * nh;
  double acc[2] = {0, 0};
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < NH; q += (size_t)gridDim.x * blockDim.x) {
    const int kz = (int)(q % nh);
    const size_t row = q / nh;
    const int kx = (int)(row / n), ky = (int)(row % n);
    const int mx = kx <= (n - 1) / 2 ? kx : kx - n, my = ky <= (n - 1) / 2 ? ky : ky - n;
    const int m2 = mx * mx + my * my + kz * kz;
    const double w = (kz == 0 || 2 * kz == n) ? 1.0 : 2.0;
    if (vloc) {
      const double G2 = tp2 * (double)m2;
      if (G2 <= g2cut) {
        const cplx<T> a = nt[q], v = vloc[q];
        const double c = m2 == 0 ? 3.0 : 1.0 - 0.5 * G2 * rc2;
        acc[0] += w * c * invN * ((double)a.x * (double)v.x + (double)a.y * (double)v.y);
      }
    }
    if (pnl) {
      const cplx<T> b = wt[q];
      acc[1] += w * invN * invN * ((double)b.x * (double)b.x + (double)b.y * (double)b.y) * pnl[m2];
    }
  }
  double o[2];
  block_sum<2>(acc, red, o);
  if (threadIdx.x == 0) { partial[(size_t)blockIdx.x * 2] = o[0]; partial[(size_t)blockIdx.x * 2 + 1] = o[1]; }
}

}  // namespace ofdft

namespace ofdft {

// The energies of a density evaluation (mode 0) from its raw sums raw[0..11]
// (see finalize_eval), written to e[0..10] in the order of ofdft_energies:
// F_TF, E_vW, E_NL, E_H, E_loc, E_xc, E_ion, F_total, N_e, mu, residual.
// One thread; the same arithmetic as the host's finish for mode 0.
static __global__ void k_finish_energies(const double* __restrict__ raw, double dV, double E_ion, int merged,
                                         double* __restrict__ e) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double E_H = raw[0], E_loc = raw[1], E_NL = raw[2], E_vW = raw[3];
  const double F_TF = raw[4] * dV, E_xc = raw[5] * dV, vn = raw[6] * dV + (merged ? E_NL : 0.0);
  const double gg = raw[8] * dV, gpsi = raw[9] * dV, ne = raw[10] * dV;
  const double mu = (vn + E_vW) / ne;
  const double r2 = (gg - 2.0 * mu * gpsi + mu * mu * ne) / ne;
  e[0] = F_TF; e[1] = E_vW; e[2] = E_NL; e[3] = E_H; e[4] = E_loc; e[5] = E_xc; e[6] = E_ion;
  e[7] = F_TF + E_vW + E_NL + E_H + E_loc + E_xc + E_ion;
  e[8] = ne; e[9] = mu; e[10] = sqrt(fmax(r2, 0.0));
}

}  // namespace ofdft
