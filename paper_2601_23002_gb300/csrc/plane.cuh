// Fused x-y transform and G-space pass over whole kz planes (plane layout).
//
// With the half spectrum stored plane by plane, [kz][kx][ky], one kz plane of
// one field (n x n complex) fits in shared memory for the grids most cells
// use (FP32 n <= 160, FP64 n <= 112).  One block then does, on data that stays
// on chip:
//   forward FFT along y, forward FFT along x, the G-space terms, inverse FFT
//   along x, inverse FFT along y
// -- the work of the y-pass / x-G-space / y-pass chain, with one read and one
// write of the spectrum instead of three of each.
//
// The transforms are in place, without a second buffer: the forward ones are
// decimation in frequency (butterfly, then twiddle), leaving the spectrum in
// mixed-radix digit-reversed order; the G-space terms only need each
// position's frequency (a table, rev[]); the inverse ones undo the forward
// stages in reverse order (conjugate twiddle, then conjugate butterfly), which
// returns natural order and the unnormalised inverse.  Every butterfly reads
// and writes its own R elements, so a stage needs no block barrier inside it.
//
// Shared memory: plane[n][n + 1] (odd row pitch: row-parallel and
// column-parallel access are both free of bank conflicts) | tw[n] | rev[n].
#pragma once
#include <cooperative_groups.h>
#include "passes.cuh"

namespace ofdft {

// One in-place stage of radix R over `lines` transforms of length n stored at
// a + line * ld_line + i * ld_elem.  The stage splits each block of Lsub
// consecutive (transform-)positions into R interleaved pieces of m = Lsub / R.
// DIR < 0: decimation in frequency, y_k = w_Lsub^(j k) DFT_R(x)_k stored at
// position j + k m of the block.  DIR > 0: the inverse of that map times R.
// line_fastest maps consecutive threads to consecutive lines.
template <typename T, int R, int DIR>
__device__ __forceinline__ void ip_stage(cplx<T>* __restrict__ a, int n, int Lsub, int ld_elem, int ld_line,
                                         int lines, bool line_fastest, const cplx<T>* __restrict__ tw) {
  const int m = Lsub / R;
  const int per_line = n / R;
  const int items = per_line * lines;            // <= 160 * 80
  const int tstep = n / Lsub;
  const unsigned Mm = qmagic(m), Mpl = qmagic(per_line), Mli = qmagic(lines);
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    int line, t;
    if (line_fastest) { t = qdiv(it, lines, Mli); line = it - t * lines; }
    else { line = qdiv(it, per_line, Mpl); t = it - line * per_line; }
    const int b = qdiv(t, m, Mm), j = t - b * m;
    // 32-bit offsets: a plane has at most 160 x 161 elements
    const int base = line * ld_line + (b * Lsub + j) * ld_elem;
    const int st = m * ld_elem;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = a[base + r * st];
    // m == 1 (the last forward / first inverse stage): j = 0, every twiddle is 1
    if (DIR > 0 && m > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = tw[j * r * tstep];             // j r < Lsub, so the index is < n
        w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    Codelet<cplx<T>, R, DIR>::run(v);
    if (DIR < 0 && m > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[j * r * tstep]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) a[base + r * st] = v[r];
  }
}

// Stage dispatch over the radices in MASK (bit r set: radix r compiled in).
// A kernel holds only the codelets its grid size uses: with all eleven
// radices inlined, a block of 16 warps stalled on instruction fetch after
// every stage barrier.
constexpr unsigned kAllRadices = (1u << 2) | (1u << 3) | (1u << 4) | (1u << 5) | (1u << 6) | (1u << 8) |
                                 (1u << 9) | (1u << 10) | (1u << 12) | (1u << 15) | (1u << 16);
template <typename T, int DIR, unsigned MASK>
__device__ __forceinline__ void ip_stage_any(int R, cplx<T>* a, int n, int Lsub, int ld_elem, int ld_line, int lines,
                                             bool line_fastest, const cplx<T>* tw) {
#define OFDFT_IP_CASE(RR)                                                              \
  if constexpr (((MASK >> RR) & 1u) != 0) {                                           \
    if (R == RR) { ip_stage<T, RR, DIR>(a, n, Lsub, ld_elem, ld_line, lines, line_fastest, tw); return; } \
  }
  OFDFT_IP_CASE(16)
  OFDFT_IP_CASE(8)
  OFDFT_IP_CASE(12)
  OFDFT_IP_CASE(10)
  OFDFT_IP_CASE(9)
  OFDFT_IP_CASE(6)
  OFDFT_IP_CASE(5)
  OFDFT_IP_CASE(4)
  OFDFT_IP_CASE(3)
  OFDFT_IP_CASE(2)
  OFDFT_IP_CASE(15)
#undef OFDFT_IP_CASE
}

// bit mask of the radices of a plan
inline unsigned radix_mask(const FftPlan1& p) {
  unsigned m = 0;
  for (int i = 0; i < p.npass; ++i) m |= 1u << p.radix[i];
  return m;
}

// Forward (DIR < 0, stages in plan order) or inverse (DIR > 0, reverse order)
// transforms of all n lines of the plane along one axis.  Ends with a barrier.
template <typename T, int DIR, unsigned MASK>
__device__ __forceinline__ void ip_fft_axis(cplx<T>* a, const FftPlan1& p, int ld_elem, int ld_line, bool rows,
                                            const cplx<T>* tw) {
  const int n = p.n;
  int Ls[8];
  int Lsub = n;
  for (int s = 0; s < p.npass; ++s) { Ls[s] = Lsub; Lsub /= p.radix[s]; }
  for (int q = 0; q < p.npass; ++q) {
    const int s = DIR < 0 ? q : p.npass - 1 - q;
    const int R = p.radix[s];
    // along rows (unit stride) keep unit-stride runs when they span a warp;
    // otherwise put consecutive threads on consecutive lines
    const bool line_fastest = !rows || Ls[s] / R < 32;
    ip_stage_any<T, DIR, MASK>(R, a, n, Ls[s], ld_elem, ld_line, n, line_fastest, tw);
    __syncthreads();
  }
}

// As ip_fft_axis, over `lines` lines (a part of the plane).
template <typename T, int DIR, unsigned MASK>
__device__ __forceinline__ void ip_fft_axis_lines(cplx<T>* a, const FftPlan1& p, int ld_elem, int ld_line,
                                                  bool rows, int lines, const cplx<T>* tw) {
  const int n = p.n;
  int Ls[8];
  int Lsub = n;
  for (int s = 0; s < p.npass; ++s) { Ls[s] = Lsub; Lsub /= p.radix[s]; }
  for (int q = 0; q < p.npass; ++q) {
    const int s = DIR < 0 ? q : p.npass - 1 - q;
    const int R = p.radix[s];
    const bool line_fastest = !rows || Ls[s] / R < 32;
    ip_stage_any<T, DIR, MASK>(R, a, n, Ls[s], ld_elem, ld_line, lines, line_fastest, tw);
    __syncthreads();
  }
}

// One in-place stage (as ip_stage) along columns of a plane whose rows are
// split between the two blocks of a cluster: row r lives in part[r / half] at
// offset (r % half) * pitch, part 0 = p0, part 1 = p1.  Transforms the ncols
// columns col0 .. col0+ncols-1.
template <typename T, int R, int DIR>
__device__ __forceinline__ void ip_stage_cols2(cplx<T>* p0, cplx<T>* p1, int half, int pitch, int n, int Lsub,
                                               int col0, int ncols, const cplx<T>* __restrict__ tw) {
  const int m = Lsub / R;
  const int items = (n / R) * ncols;
  const int tstep = n / Lsub;
  const unsigned Mm = qmagic(m), Mc = qmagic(ncols);
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int t = qdiv(it, ncols, Mc), col = col0 + (it - t * ncols);
    const int b = qdiv(t, m, Mm), j = t - b * m;
    const int row0 = b * Lsub + j;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = row0 + r * m;
      const bool hi = row >= half;
      v[r] = (hi ? p1 : p0)[(row - (hi ? half : 0)) * pitch + col];
    }
    if (DIR > 0 && m > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = tw[j * r * tstep];
        w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    Codelet<cplx<T>, R, DIR>::run(v);
    if (DIR < 0 && m > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[j * r * tstep]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = row0 + r * m;
      const bool hi = row >= half;
      (hi ? p1 : p0)[(row - (hi ? half : 0)) * pitch + col] = v[r];
    }
  }
}

template <typename T, int DIR, unsigned MASK>
__device__ __forceinline__ void ip_stage_cols2_any(int R, cplx<T>* p0, cplx<T>* p1, int half, int pitch, int n,
                                                   int Lsub, int col0, int ncols, const cplx<T>* tw) {
#define OFDFT_IP2_CASE(RR)                                                                \
  if constexpr (((MASK >> RR) & 1u) != 0) {                                              \
    if (R == RR) { ip_stage_cols2<T, RR, DIR>(p0, p1, half, pitch, n, Lsub, col0, ncols, tw); return; } \
  }
  OFDFT_IP2_CASE(16)
  OFDFT_IP2_CASE(8)
  OFDFT_IP2_CASE(12)
  OFDFT_IP2_CASE(10)
  OFDFT_IP2_CASE(9)
  OFDFT_IP2_CASE(6)
  OFDFT_IP2_CASE(5)
  OFDFT_IP2_CASE(4)
  OFDFT_IP2_CASE(3)
  OFDFT_IP2_CASE(2)
  OFDFT_IP2_CASE(15)
#undef OFDFT_IP2_CASE
}

constexpr int kPlaneThreads = 512;

// grid.x = kz plane (n/2 + 1), grid.y = active field.  Spectra in plane
// layout: field f's plane kz is sp.s[f] + kz * n * n, row kx, column ky.
// vloc (if given) is in plane layout and position order: entry (kz, px, py)
// is V_loc(kx = rev[px], ky = rev[py], kz).
template <typename T, unsigned MASK>
__global__ void __launch_bounds__(kPlaneThreads, 1) k_plane(Spectra<T> sp, GArgs<T> g, FftPlan1 pn,
                                                            const int* __restrict__ rev_g,
                                                            const cplx<T>* __restrict__ tw_g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = pn.n, pitch = n + 1, nn = n * n;
  cplx<T>* a = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tw = a + (size_t)n * pitch;
  int* rev = reinterpret_cast<int*>(tw + n);
  const int kz = blockIdx.x;
  const int fid = sp.idx[blockIdx.y];
  cplx<T>* gpl = sp.s[fid] + (size_t)kz * nn;
  const unsigned Mn = qmagic(n);
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const int r = qdiv(q, n, Mn), c = q - r * n;
    cp_async_c(a + r * pitch + c, gpl + q, true);
  }
  cp_async_commit();
  for (int q = threadIdx.x; q < n; q += blockDim.x) { tw[q] = tw_g[q]; rev[q] = rev_g[q]; }
  cp_async_wait<0>();
  __syncthreads();
  ip_fft_axis<T, -1, MASK>(a, pn, 1, pitch, true, tw);       // along ky (rows)
  ip_fft_axis<T, -1, MASK>(a, pn, pitch, 1, false, tw);      // along kx (columns)
  // G-space terms (same arithmetic as the x/G-space pass of the tiled path)
  const T tp2 = g.tp2, invN = g.invN, Om = g.Om, halfOm = g.halfOm, fourpi = (T)(4.0 * kPi);
  const T g2cut = g.g2cut_loc;
  const bool with_loc = fid == 0 && g.vloc != nullptr;
  const T w = (kz == 0 || 2 * kz == n) ? (T)1 : (T)2;
  const cplx<T>* vpl = with_loc ? g.vloc + (size_t)kz * nn : nullptr;
  AccShort<T> acc[4];
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const int px = qdiv(q, n, Mn), py = q - px * n;
    const int kx = rev[px], ky = rev[py];
    const int mx = kx <= (n - 1) / 2 ? kx : kx - n;
    const int my = ky <= (n - 1) / 2 ? ky : ky - n;
    const int m2 = mx * mx + my * my + kz * kz;
    const T G2 = tp2 * (T)m2;
    cplx<T>* cell = a + px * pitch + py;
    const cplx<T> v = *cell;
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
      if (with_loc && G2 <= g2cut) {            // zero beyond the cutoff
        const cplx<T> vl = vpl[q];
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
    *cell = o;
  }
  __syncthreads();
  ip_fft_axis<T, 1, MASK>(a, pn, pitch, 1, false, tw);       // inverse along kx
  ip_fft_axis<T, 1, MASK>(a, pn, 1, pitch, true, tw);        // inverse along ky
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const int r = qdiv(q, n, Mn), c = q - r * n;
    gpl[q] = a[r * pitch + c];
  }
  const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
  block_sum_tree_raw<4, T>(acc, g.partials + b * 4, reinterpret_cast<typename TreeVal<T>::type*>(smem_raw));
}

// The one-field preconditioning pass (out = IFFT[p(G) FFT(in)], GArgs::prec)
// on one kz plane per cluster of two blocks: block `rank` holds rows
// rank*n/2 .. rank*n/2 + n/2 - 1 of the plane (half the shared memory of
// k_plane); the transforms along rows are local, those along columns split the
// columns between the pair and reach the partner's rows through distributed
// shared memory, with a cluster barrier after every stage.  With one field the
// plain plane pass occupies only n/2 + 1 SMs; this uses twice as many, each
// with half the work.  grid.x = 2 (n/2 + 1).
template <typename T, unsigned MASK>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPlaneThreads, 1)
k_plane_prec2(Spectra<T> sp, GArgs<T> g, FftPlan1 pn, const int* __restrict__ rev_g,
              const cplx<T>* __restrict__ tw_g) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = pn.n, pitch = n + 1, half = n / 2, nn = n * n;
  const int rank = (int)cl.block_rank();
  cplx<T>* a = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tw = a + (size_t)half * pitch;
  int* rev = reinterpret_cast<int*>(tw + n);
  cplx<T>* const p0 = rank == 0 ? a : cl.map_shared_rank(a, 0);   // rows 0 .. n/2 - 1
  cplx<T>* const p1 = rank == 1 ? a : cl.map_shared_rank(a, 1);   // rows n/2 .. n - 1
  const int kz = blockIdx.x >> 1;
  const int fid = sp.idx[0];
  cplx<T>* gpl = sp.s[fid] + (size_t)kz * nn + (size_t)rank * half * n;   // this block's rows
  const unsigned Mn = qmagic(n);
  for (int q = threadIdx.x; q < half * n; q += blockDim.x) {
    const int r = qdiv(q, n, Mn), c = q - r * n;
    cp_async_c(a + r * pitch + c, gpl + q, true);
  }
  cp_async_commit();
  for (int q = threadIdx.x; q < n; q += blockDim.x) { tw[q] = tw_g[q]; rev[q] = rev_g[q]; }
  cp_async_wait<0>();
  __syncthreads();
  ip_fft_axis_lines<T, -1, MASK>(a, pn, 1, pitch, true, half, tw);   // along ky, own rows
  cl.sync();
  int Ls[8];
  {
    int Lsub = n;
    for (int s = 0; s < pn.npass; ++s) { Ls[s] = Lsub; Lsub /= pn.radix[s]; }
  }
  for (int q = 0; q < pn.npass; ++q) {                                 // along kx, half the columns
    ip_stage_cols2_any<T, -1, MASK>(pn.radix[q], p0, p1, half, pitch, n, Ls[q], rank * half, half, tw);
    cl.sync();
  }
  // p(G) f~(G) on own rows
  const T invN = g.invN;
  for (int q = threadIdx.x; q < half * n; q += blockDim.x) {
    const int r = qdiv(q, n, Mn), py = q - r * n;
    const int px = rank * half + r;
    const int kx = rev[px], ky = rev[py];
    const int mx = kx <= (n - 1) / 2 ? kx : kx - n;
    const int my = ky <= (n - 1) / 2 ? ky : ky - n;
    const int m2 = mx * mx + my * my + kz * kz;
    cplx<T>* cell = a + r * pitch + py;
    const cplx<T> v = *cell;
    const T vr = v.x * invN, vi = v.y * invN;   // as k_plane: the same bits
    const T pg = g.prec[m2];
    *cell = mk<T>(pg * vr, pg * vi);
  }
  cl.sync();
  for (int q = 0; q < pn.npass; ++q) {                                 // inverse along kx
    const int st = pn.npass - 1 - q;
    ip_stage_cols2_any<T, 1, MASK>(pn.radix[st], p0, p1, half, pitch, n, Ls[st], rank * half, half, tw);
    cl.sync();                                                         // (last: no remote access after)
  }
  ip_fft_axis_lines<T, 1, MASK>(a, pn, 1, pitch, true, half, tw);    // inverse along ky, own rows
  for (int q = threadIdx.x; q < half * n; q += blockDim.x) {
    const int r = qdiv(q, n, Mn), c = q - r * n;
    gpl[q] = a[r * pitch + c];
  }
}

// The plane kernel compiled for a plan's radices (instantiated in
// plane_f32.cu / plane_f64.cu for the radix sets of the supported grids; any
// other set gets the kernel with every radix).
template <typename T>
using PlaneKernel = void (*)(Spectra<T>, GArgs<T>, FftPlan1, const int*, const cplx<T>*);
template <typename T> PlaneKernel<T> plane_kernel(unsigned mask);
template <typename T> PlaneKernel<T> plane_prec2_kernel(unsigned mask);

// One-time reorder of V_loc from the tiled layout [kx][ky][kz] into plane
// layout and position order: dst[(kz n + px) n + py] = src[(rev[px] n + rev[py]) nh + kz].
template <typename T>
__global__ void k_vloc_planes(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst,
                              const int* __restrict__ rev, int n) {
  const int nh = n / 2 + 1;
  const size_t tot = (size_t)nh * n * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    const int py = (int)(i % n);
    const int px = (int)((i / n) % n);
    const int kz = (int)(i / ((size_t)n * n));
    dst[i] = src[((size_t)rev[px] * n + rev[py]) * nh + kz];
  }
}

}  // namespace ofdft
