// Per-precision engine: device buffers of one plan, the evaluation pipeline,
// setup, S_ei, and the L-BFGS driver.  Included by engine_f32.cu / engine_f64.cu.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "engine.h"
#include "profiler.h"
#include "fft.cuh"
#include "passes.cuh"
#include "plane.cuh"
#include "setup.cuh"
#include "vecops.cuh"
#include "zpass256.cuh"

namespace ofdft {

#define OFDFT_CK(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      set_error(std::string("CUDA error: ") + cudaGetErrorString(e_) + " at " + #call); \
      return e_ == cudaErrorMemoryAllocation ? OFDFT_ERR_OOM : OFDFT_ERR_CUDA;          \
    }                                                                                   \
  } while (0)

#define OFDFT_LAUNCH_CK()                                                               \
  do {                                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess) {                                                            \
      set_error(std::string("CUDA launch error: ") + cudaGetErrorString(e_));           \
      return OFDFT_ERR_CUDA;                                                            \
    }                                                                                   \
  } while (0)

#define OFDFT_RUN(name, st, bytes, ...)  \
  do {                            \
    prof.begin(name, st, (double)(bytes)); \
    __VA_ARGS__;                  \
    prof.end(st);                 \
    OFDFT_LAUNCH_CK();            \
  } while (0)

constexpr int kThreads = 256;

template <typename T>
__global__ void k_convert_table(const double* __restrict__ a, T* __restrict__ b, int cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) b[i] = (T)a[i];
}
constexpr int kMaxMem = 16;
// res_d / res_h: 0..13 evaluation, 16..119 Gram and direction dots, 120..125
// k_accept's dots, 126..128 the device-formed trial (scale, psi shift, t),
// 129..130 the device recursion's gamma and pairs used
constexpr int kResSlots = 160;

// ring slot of the i-th oldest history pair
struct Ring {
  int head = 0, count = 0, m = 8;
  int slot(int i) const { return (head + i) % m; }   // i = 0 oldest
  int push() {                                      // returns slot for the new pair
    int s;
    if (count < m) { s = (head + count) % m; ++count; }
    else { s = head; head = (head + 1) % m; }
    return s;
  }
  void clear() { head = 0; count = 0; }
};

template <typename T>
class Engine : public IEngine {
 public:
  using C = cplx<T>;
  CellSpec cs;
  int n = 0, nh = 0, h = 0;
  size_t N = 0, NH = 0;
  // length of the minimiser's vectors: N rounded up to whole 16-byte groups
  // of the streaming passes (odd n); the padding is zero and stays zero
  size_t Nv = 0;
  double L = 0, Omega = 0, dV = 0, Ne = 0, nbar = 0, Te = 0;
  int m_max = 8;
  FftPlan1 pn{}, ph{};
  // launch geometry
  int zR = 0, zP = 0, yJ = 0, xJ = 0;
  size_t smem_zf = 0, smem_zi = 0, smem_y = 0, smem_x = 0, smem_xp = 0;
  // n = 256, FP32, tiled path: the z passes with register transforms (zpass256.cuh)
  bool z256 = false, z256_allowed = true;
  size_t smem_zf256 = 0, smem_zi256 = 0;
  // and the cluster plane pass of that grid (spectra in plane layout;
  // OFDFT_P256=0 keeps the tiled register passes)
  bool p256 = false, p256_allowed = true;
  // and the y and x/G-space passes of that grid (16-column tiles)
  static constexpr int kGridY256 = 256 * 9, kGridX256 = 256 * 129 / 16;
  int grid_z = 0, grid_y1 = 0, grid_x = 0, grid_vec = 0, grid_stream = 0, nsm = 152;
  // device memory
  std::vector<std::pair<void*, size_t>> allocs;   // (block, bytes) from the block cache
  size_t nbytes = 0;
  C *tw_n = nullptr, *tw_h = nullptr;
  double* Kd = nullptr;
  double2* sf_tab = nullptr;   // per m^2: (v~/Omega per unit charge, Ewald reciprocal weight)
  T* Kt = nullptr;
  C* vloc = nullptr;
  C* Sg = nullptr;
  C* SZg = nullptr;          // S_Z(G) = sum_I Z_I exp(-i G.R_I), tiled layout (forces)
  // plane path (fused x-y-G-space pass; spectra in plane layout) when a kz
  // plane fits in shared memory
  bool plane_allowed = true;
  bool planes = false;
  size_t smem_pl = 0;
  int* rev_d = nullptr;      // position -> frequency of the in-place transforms
  PlaneKernel<T> plane_kern = nullptr;   // k_plane compiled for this grid's radices
  // one-field preconditioning pass on two-block clusters (half a plane per
  // block) when half a plane fits in shared memory
  bool prec2 = false, prec2_allowed = true;
  size_t smem_pl2 = 0;
  PlaneKernel<T> prec2_kern = nullptr;
  // V_loc in plane layout: position order for the plane pass, natural order
  // [kz][kx][ky] for the 256^3 cluster plane pass
  C* vloc_pl = nullptr;
  C* spec[3] = {nullptr, nullptr, nullptr};
  T *psi = nullptr, *d = nullptr, *g = nullptr, *gp = nullptr;
  // preconditioned two-loop recursion: P g (current and previous g), P y of
  // the history pairs, and the table p(m^2)
  T* pgv[2] = {nullptr, nullptr};
  T* PYh[kMaxMem] = {};
  T* precT = nullptr;
  T* Sh[kMaxMem] = {};
  T* Yh[kMaxMem] = {};
  double* partials = nullptr;
  size_t partials_cap = 0;
  double* res_d = nullptr;
  TwoLoopState* tl_state = nullptr;   // L-BFGS history scalars on the device
  double* res_h = nullptr;     // pinned
  unsigned int* counters = nullptr;   // last-block arrival counters (0 between launches)
  double* pos_d = nullptr;
  double* Z_d = nullptr;
  double2* phases = nullptr;
  double E_ion = 0;
  bool ions_set = false;
  double g2cut_loc = 0;
  // Ewald splitting of the last set_ions, reused by forces
  double ew_eta = 0, ew_rcut = 0;
  int ew_nimg = 0;
  // forces: G list {kx, ky, kz, w} with 0 < |G|^2 <= g2cut_loc, its (vfac, efac),
  // per-G weights qq, ion phases in T, device output; built on the first call
  int4* f_gl = nullptr;
  double2* f_gf = nullptr;
  C* f_qq = nullptr;
  C* f_pt = nullptr;
  double* f_out = nullptr;
  int f_ng = -1;
  // pressure: pnl(m^2) = (3 - 6a) K + dK/dlambda (FP64, built on the first call)
  double* p_tab = nullptr;
  bool p_ready = false;
  // |q| shells of the structure factors: CSR lists of half-spectrum entries
  // with Hermitian weights, kept for the last n_shells asked for
  int sh_ns = 0;
  long long sh_entries = 0;
  std::vector<int> sh_m2;
  int* sh_ptr = nullptr;
  long long* sh_idx = nullptr;
  float* sh_w = nullptr;
  double* sh_out = nullptr;
  size_t sh_bytes[4] = {0, 0, 0, 0};
  void free_shells() {
    void* p[4] = {sh_ptr, sh_idx, sh_w, sh_out};
    for (int i = 0; i < 4; ++i) cached_dev_release(p[i], sh_bytes[i]);
    sh_ptr = nullptr; sh_idx = nullptr; sh_w = nullptr; sh_out = nullptr; sh_ns = 0;
  }
  size_t n_vloc = 0;         // half-spectrum entries with |G|^2 <= g2cut_loc
  double mean_params[4] = {0, 0, 0, 0};
  Profiler prof;
  struct Tune { int zR = 0, yJ = 0, xJ = 0; } tune;   // launch-shape overrides (0 = default)

  explicit Engine(const CellSpec& c, int mmax) : cs(c), m_max(mmax) {
    auto env = [](const char* k) { const char* v = std::getenv(k); return v ? std::atoi(v) : 0; };
    tune.zR = env("OFDFT_ZR");
    const char* pe = std::getenv("OFDFT_PLANE");
    plane_allowed = !(pe && pe[0] == '0');
    const char* z2 = std::getenv("OFDFT_Z256");
    z256_allowed = !(z2 && z2[0] == '0');
    const char* q2 = std::getenv("OFDFT_P256");
    p256_allowed = !(q2 && q2[0] == '0');
    const char* p2 = std::getenv("OFDFT_PREC2");
    prec2_allowed = !(p2 && p2[0] == '0');
    tune.yJ = env("OFDFT_YJ");
    tune.xJ = env("OFDFT_XJ");
  }
  ~Engine() override {
    // the blocks go back to the cache once work queued without a synchronising
    // return has drained (a stream that no longer exists: the whole device)
    for (void* s : async_streams)
      if (cudaStreamSynchronize((cudaStream_t)s) != cudaSuccess) {
        cudaGetLastError();
        cudaDeviceSynchronize();
      }
    for (auto& a : allocs) cached_dev_release(a.first, a.second);
    free_shells();
    cached_host_release(res_h, kResSlots * sizeof(double));
  }
  size_t bytes() const override { return nbytes; }
  int profile_enable(int timing) override { prof.reset(timing != 0); return OFDFT_OK; }
  int profile_read(ofdft_kernel_stat* out, int max, int* count) override {
    const auto& st = prof.stats();
    int i = 0;
    for (const auto& kv : st) {
      if (out && i < max) {
        std::memset(out[i].name, 0, sizeof(out[i].name));
        std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
        out[i].launches = kv.second.launches;
        out[i].total_ms = kv.second.ms;
        out[i].bytes = kv.second.bytes;
      }
      ++i;
    }
    if (count) *count = i;
    return OFDFT_OK;
  }

  template <typename P> int alloc(P** p, size_t count) {
    void* q = nullptr;
    const size_t b = count * sizeof(P);
    const size_t bb = b > 0 ? (b + 255) / 256 * 256 : 256;   // sizes in 256-byte steps, for reuse
    cudaError_t e = cached_dev_alloc(&q, bb);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("device allocation of ") + std::to_string(b) + " bytes failed: " +
                cudaGetErrorString(e));
      return OFDFT_ERR_OOM;
    }
    allocs.push_back({q, bb});
    nbytes += b;
    *p = reinterpret_cast<P*>(q);
    return OFDFT_OK;
  }

  bool use_n() const { return (cs.terms & (OFDFT_TERM_HARTREE | OFDFT_TERM_LOC)) != 0; }
  bool use_na() const { return (cs.terms & OFDFT_TERM_NL) != 0; }
  bool use_psi() const { return (cs.terms & OFDFT_TERM_VW) != 0; }

  // a = 1/2 with vW and NL both on: one psi spectrum serves both terms
  bool merged() const { return use_na() && use_psi() && cs.alpha == 0.5; }

  Spectra<T> spectra() const {
    Spectra<T> s{};
    s.nact = 0;
    s.merged = merged() ? 1 : 0;
    s.planes = (planes || p256) ? 1 : 0;
    const bool on[3] = {use_n(), use_na() && !merged(), use_psi()};
    for (int f = 0; f < 3; ++f) {
      s.s[f] = on[f] ? spec[f] : nullptr;
      if (on[f]) s.idx[s.nact++] = f;
    }
    return s;
  }

  static size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

  // epilogue pass: staging of the active spectra, two FFT buffers, the block's
  // rho or psi and d rows
  size_t zinv_bytes(int r) const {
    const int nact = spectra().nact;
    return (size_t)nact * r * (n / 2 + 1) * sizeof(C) + 2 * zbuf_elems(n, r, zpitch()) * sizeof(C) +
           2 * (size_t)r * n * sizeof(T);
  }
  // row pitch of the z passes' FFT buffers: odd and >= the transform length
  // (n / 2 + 1 half-length rows for even n; length-n rows of two packed real
  // rows for odd n)
  int zpitch() const { return (n & 1) ? n : ((n / 2 + 1) | 1); }

  void geometry() {
    n = cs.n; h = n / 2; nh = h + 1;
    N = (size_t)n * n * n;
    NH = (size_t)n * n * nh;
    Nv = (N + 3) & ~(size_t)3;
    L = cs.L; Omega = L * L * L; dV = Omega / (double)N;
    Ne = 0; for (double z : cs.Z) Ne += z;
    nbar = Ne / Omega; Te = cs.T;
    zR = std::max(1, std::min(16, 1024 / h));     // 16 rows per block: best in a sweep at 128^3
    zP = zpitch();
    yJ = sizeof(T) == 4 ? 16 : 8;
    xJ = yJ;
    // overrides (autotuner, set_tiles, OFDFT_ZR/YJ/XJ) only within the shapes
    // the reduction scratch was sized for: at least 8 rows / 8 columns
    if (tune.zR >= 8 && tune.zR <= 64) zR = tune.zR;
    // odd n: the z passes pair rows, and an even row count keeps every
    // block's rows on an 8-byte boundary
    if (n & 1) zR = std::max(2, zR & ~1);
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    if (tune.yJ >= 8 && tune.yJ <= 64 && pow2(tune.yJ)) yJ = tune.yJ;
    if (tune.xJ >= 8 && tune.xJ <= 64 && pow2(tune.xJ)) xJ = tune.xJ;
    smem_zf = align16((size_t)2 * zR * n * sizeof(T)) + 2 * zbuf_elems(n, zR, zP) * sizeof(C);
    // (the G-space and epilogue passes reuse their tiles as reduction scratch)
    smem_zi = std::max(zinv_bytes(zR), tree_scratch_bytes<T>(12, kThreads));   // finalize: 12 columns
    smem_y = 2 * (size_t)n * yJ * sizeof(C);
    smem_x = std::max(3 * (size_t)n * xJ * sizeof(C), tree_scratch_bytes<T>(4, kThreads));
    smem_xp = 2 * (size_t)n * xJ * sizeof(C);
    grid_z = (int)(((size_t)n * n + zR - 1) / zR);
    grid_y1 = n * ((nh + yJ - 1) / yJ);
    grid_x = (int)(((size_t)n * nh + xJ - 1) / xJ);
    smem_pl = std::max(((size_t)n * (n + 1) + n) * sizeof(C) + (size_t)n * sizeof(int),
                       tree_scratch_bytes<T>(4, kPlaneThreads));
    planes = plane_allowed && smem_pl <= (size_t)225 * 1024;
    // (rows per block even and dividing n^2: 8, 16 or 32)
    z256 = z256_allowed && sizeof(T) == 4 && n == 256 && !planes && (zR == 8 || zR == 16 || zR == 32);
    p256 = z256 && p256_possible();
    smem_zf256 = z256_fwd_bytes<T>(zR);
    smem_zi256 = std::max(z256_inv_bytes<T>(zR, spectra().nact), tree_scratch_bytes<T>(12, kThreads));
    // clusters only for large grids: below n = 112 the snapshots that are
    // solved side by side (batched, served) fill the GPU anyway, and a
    // cluster launch waits for pairs of free SMs (64 cells of 48^3-96^3:
    // 712 -> 669 snapshots/s with clusters)
    smem_pl2 = ((size_t)(n / 2) * (n + 1) + n) * sizeof(C) + (size_t)n * sizeof(int);
    // (even n only: the pair splits the plane's rows in two equal halves)
    prec2 = plane_allowed && prec2_allowed && n >= 112 && n % 2 == 0 && smem_pl2 <= (size_t)225 * 1024;
    // streaming vector kernels: a multiple of the SM count (4 resident blocks
    // per SM); the async-copy ring kernels hold 160 KB of shared memory, one
    // block per SM
    grid_vec = (int)std::min<size_t>((size_t)4 * nsm, (N + kThreads - 1) / kThreads);
    grid_stream = (int)std::min<size_t>((size_t)nsm, (Nv / StreamCfg<T>::K + kStreamThreads - 1) / kStreamThreads);
  }

  // the cluster plane pass at 256^3 for some row count (V_loc in its order is
  // then kept whatever the tiles)
  // the z passes at 256^3 for the plan's rows per block (FP32 plans)
  int launch_zfwd256(const ProArgs<T>& pa, const Spectra<T>& sp, double bytes, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
      auto k = zR == 8 ? k_zfwd256<T, 8> : (zR == 16 ? k_zfwd256<T, 16> : k_zfwd256<T, 32>);
      OFDFT_RUN("k_zfwd256", st, bytes, k<<<grid_z, kThreads, smem_zf256, st>>>(pa, sp, tw_h, tw_n));
      return OFDFT_OK;
    } else {
      set_error("the 256^3 register z passes are FP32 only");
      return OFDFT_ERR_INVALID;
    }
  }
  int launch_zinv256(const Spectra<T>& sp, const EpiArgs<T>& ea, double bytes, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
      auto k = zR == 8 ? k_zinv256<T, 8> : (zR == 16 ? k_zinv256<T, 16> : k_zinv256<T, 32>);
      OFDFT_RUN("k_zinv256", st, bytes, k<<<grid_z, kThreads, smem_zi256, st>>>(sp, ea, tw_h, tw_n));
      return OFDFT_OK;
    } else {
      set_error("the 256^3 register z passes are FP32 only");
      return OFDFT_ERR_INVALID;
    }
  }

  bool p256_possible() const { return z256_allowed && p256_allowed && sizeof(T) == 4 && n == 256 && !planes; }

  // the cluster plane pass over nf fields
  int launch_p256(const Spectra<T>& sp, const GArgs<T>& ga, int nf, double bytes, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
      OFDFT_RUN("k_plane256cl", st, bytes, k_plane256cl<T><<<dim3(P256::CL * nh, nf), P256::THREADS, p256_bytes<T>(), st>>>(sp, ga, tw_n));
      return OFDFT_OK;
    } else {
      set_error("the cluster plane pass is FP32 only");
      return OFDFT_ERR_INVALID;
    }
  }

  size_t plan_bytes_estimate() {
    geometry();
    size_t b = 0;
    b += 3 * NH * sizeof(C) + 2 * NH * sizeof(C);           // spectra, vloc, S
    if (planes || p256_possible()) b += NH * sizeof(C);      // vloc in plane order
    b += (6 + 3 * (size_t)m_max) * ((Nv * sizeof(T) + 255) / 256 * 256);   // psi d g gp, P g x2, history s y P y
    b += (size_t)(3 * (n / 2) * (n / 2) + 1) * (sizeof(double) + sizeof(T));
    b += (size_t)(n + h) * sizeof(C);
    return b;
  }

  int create(void* stream_) override {
    cudaStream_t st = (cudaStream_t)stream_;
    {
      int dev = 0;
      if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (nsm < 1) nsm = 152;
    }
    geometry();
    // (64-point halves at 128^3: radices 8, 8 rather than 16, 4 -- 128 butterflies per stage for a
    // 16-row block instead of 64 in the radix-16 stage; z passes measured 1-2% faster)
    if (!factor_radices(n, pn.radix, &pn.npass) || (n % 2 == 0 && !factor_radices_balanced(h, ph.radix, &ph.npass))) {
      set_error("grid size not supported by the FFT radices");
      return OFDFT_ERR_INVALID;
    }
    pn.n = n; ph.n = h;
    // odd n: the z passes transform pairs of real rows at full length
    const int nzt = (n & 1) ? n : h;          // length of the z passes' transforms
    if (n & 1) ph = pn;
    if (const char* zr = (n & 1) ? nullptr : std::getenv("OFDFT_ZRADIX")) {
      // override of the z passes' half-length radices for tuning, e.g. "8,8"
      // (used only if they are supported and multiply to n/2)
      FftPlan1 q{};
      q.n = h;
      int prod = 1;
      for (const char* c = zr; *c && q.npass < 8;) {
        const int r = std::atoi(c);
        if (r != 2 && r != 3 && r != 4 && r != 5 && r != 6 && r != 8 && r != 9 && r != 10 && r != 12 &&
            r != 15 && r != 16) { prod = -1; break; }
        q.radix[q.npass++] = r;
        prod *= r;
        while (*c && *c != ',') ++c;
        if (*c == ',') ++c;
      }
      if (prod == h) ph = q;
    }
    if (planes) plane_kern = plane_kernel<T>(radix_mask(pn));
    if (prec2) prec2_kern = plane_prec2_kernel<T>(radix_mask(pn));
    int rc;
    // twiddles
    std::vector<C> twn(n), twh(nzt);
    for (int t = 0; t < n; ++t) {
      long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)t / (long double)n;
      twn[t] = mk<T>((T)cosl(a), (T)sinl(a));
    }
    for (int t = 0; t < nzt; ++t) {
      long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)t / (long double)nzt;
      twh[t] = mk<T>((T)cosl(a), (T)sinl(a));
    }
    if ((rc = alloc(&tw_n, n))) return rc;
    if ((rc = alloc(&tw_h, nzt))) return rc;
    OFDFT_CK(cudaMemcpyAsync(tw_n, twn.data(), n * sizeof(C), cudaMemcpyHostToDevice, st));
    OFDFT_CK(cudaMemcpyAsync(tw_h, twh.data(), nzt * sizeof(C), cudaMemcpyHostToDevice, st));
    // buffers
    for (int f = 0; f < 3; ++f)
      if ((rc = alloc(&spec[f], NH))) return rc;
    if ((rc = alloc(&vloc, NH))) return rc;
    if ((rc = alloc(&Sg, NH))) return rc;
    if ((rc = alloc(&SZg, NH))) return rc;
    if (planes || prec2) {
      // frequency at each position after the in-place forward stages:
      // position p = sum_s k_s m_s (m_s = block length / R_s at stage s)
      // holds frequency sum_s k_s R_1 ... R_(s-1)
      std::vector<int> rev(n);
      for (int p = 0; p < n; ++p) {
        int rem = p, f = 0, mult = 1, Lsub = n;
        for (int s2 = 0; s2 < pn.npass; ++s2) {
          const int m = Lsub / pn.radix[s2];
          f += (rem / m) * mult;
          rem %= m;
          mult *= pn.radix[s2];
          Lsub = m;
        }
        rev[p] = f;
      }
      if ((rc = alloc(&rev_d, n))) return rc;
      OFDFT_CK(cudaMemcpyAsync(rev_d, rev.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
      if (planes && (rc = alloc(&vloc_pl, NH))) return rc;
    }
    if (p256_possible() && (rc = alloc(&vloc_pl, NH))) return rc;
    {
      // the minimiser's 6 + 3 m vectors in one allocation (slices on
      // 256-byte boundaries): one cudaMalloc instead of thirty per plan
      T** vecs[6] = {&psi, &d, &g, &gp, &pgv[0], &pgv[1]};
      const size_t slice = (Nv * sizeof(T) + 255) / 256 * 256 / sizeof(T);
      T* arena = nullptr;
      if ((rc = alloc(&arena, slice * (6 + 3 * (size_t)m_max)))) return rc;
      size_t k = 0;
      for (T** v : vecs) *v = arena + slice * k++;
      for (int i = 0; i < m_max; ++i) {
        Sh[i] = arena + slice * k++;
        Yh[i] = arena + slice * k++;
        PYh[i] = arena + slice * k++;
      }
      if (Nv > N) {
        // zero padding: the grid kernels write [0, N) only, the streaming
        // passes map zeros to zeros there, so the padding adds nothing to a dot
        for (T** v : vecs) OFDFT_CK(cudaMemsetAsync(*v + N, 0, (Nv - N) * sizeof(T), st));
        for (int i = 0; i < m_max; ++i) {
          OFDFT_CK(cudaMemsetAsync(Sh[i] + N, 0, (Nv - N) * sizeof(T), st));
          OFDFT_CK(cudaMemsetAsync(Yh[i] + N, 0, (Nv - N) * sizeof(T), st));
          OFDFT_CK(cudaMemsetAsync(PYh[i] + N, 0, (Nv - N) * sizeof(T), st));
        }
      }
    }
    const int nm2 = 3 * h * h + 1;
    if ((rc = alloc(&Kd, nm2))) return rc;
    if ((rc = alloc(&Kt, nm2))) return rc;
    // eval uses [0, 4 grid_x) for G-space partials and [4 grid_x, 4 grid_x + 8 grid_z) for the epilogue
    // (sized for the smallest tiles the autotuner may pick: 8 rows, 8 columns)
    partials_cap = std::max<size_t>({(size_t)grid_x * 12 + (size_t)grid_z * 8,
                                     ((size_t)n * nh + 7) / 8 * 12 + ((size_t)n * n + 7) / 8 * 8,
                                     (size_t)grid_vec * kMaxV * kMaxW, (size_t)n * n, (size_t)4096});
    if ((rc = alloc(&partials, partials_cap))) return rc;
    if ((rc = alloc(&res_d, kResSlots))) return rc;
    if ((rc = alloc(&tl_state, 1))) return rc;
    if ((rc = alloc(&counters, 8))) return rc;
    OFDFT_CK(cudaMemsetAsync(counters, 0, 8 * sizeof(unsigned int), st));
    OFDFT_CK(cudaMemsetAsync(res_d, 0, kResSlots * sizeof(double), st));
    OFDFT_CK(cached_host_alloc((void**)&res_h, kResSlots * sizeof(double)));
    if ((rc = alloc(&pos_d, (size_t)cs.Z.size() * 3))) return rc;
    if ((rc = alloc(&Z_d, cs.Z.size()))) return rc;
    if ((rc = alloc(&phases, (size_t)cs.Z.size() * 3 * n))) return rc;
    OFDFT_CK(cudaMemcpyAsync(Z_d, cs.Z.data(), cs.Z.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    // shared-memory limits
    if ((rc = raise_smem_limits())) return rc;
    // mean-density ideal gas: eta0, mu0, dmu0/dn
    const double y = 9.8696044010893586188 * nbar / (1.4142135623730950488 * pow(Te, 1.5));
    OFDFT_RUN("k_mean_density", st, 32.0, k_mean_density<<<1, kMeanThreads, 0, st>>>(y, Te, res_d));
    OFDFT_CK(cudaMemcpyAsync(res_h, res_d, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    OFDFT_CK(cudaStreamSynchronize(st));
    std::memcpy(mean_params, res_h, 4 * sizeof(double));
    if (use_na()) {
      KernArgs ka{L, nbar, Te, mean_params[1], mean_params[2], cs.alpha, nm2};
      OFDFT_RUN("k_kernel_table", st, (double)nm2 * 8, k_kernel_table<<<kernel_table_blocks(nm2), 32 * kKernWarps, 0, st>>>(ka, Kd));
    } else {
      OFDFT_CK(cudaMemsetAsync(Kd, 0, nm2 * sizeof(double), st));
    }
    OFDFT_RUN("k_convert_table", st, (double)nm2 * (8 + sizeof(T)), k_convert_table<T><<<(nm2 + 255) / 256, 256, 0, st>>>(Kd, Kt, nm2));
    {
      // preconditioner of the minimiser: p(G) = c / h(G), h(G) a model of the
      // psi-Hessian at the mean density per unit |dpsi~(G)|^2:
      //   h(G) = c + G^2/2 + f_K 4 a^2 nbar^(2a-1) K(G) + f_H 8 pi nbar / G^2.
      // c stands for the Thomas-Fermi term: its psi-Hessian at the mean
      // density is about 2 mu + 4 n dmu/dn, ~4 E_F degenerate and ~4 T
      // classical; c = 4 (E_F + T).  G^2/2 is the vW term.  The nonlocal
      // term's own curvature is its kernel K(G) (a = 1/2), and a density wave
      // dn = 2 sqrt(nbar) dpsi costs the Hartree energy (Omega/2) 4 pi
      // |dn~|^2 / G^2, i.e. 8 pi nbar / G^2: in large cells this long-wavelength
      // stiffness exceeds c at the smallest G (the 58.6-bohr 1024-ion cell:
      // 22 c) and set the iteration count (131 evaluations without it).
      // f_K = 1 and f_H = 1.5 (and the factor 4 of c) were the best of a scan
      // over the 256^3 and 128^3 single cells, 16 batched and 17 served cells
      // (68, 10, 254 and 230 evaluations); OFDFT_PREC_C, OFDFT_PREC_H and
      // OFDFT_PREC_K replace the three factors, for such studies.
      const double kF = std::cbrt(3.0 * kPi * kPi * nbar);
      double cfac = 4.0;
      if (const char* ev = std::getenv("OFDFT_PREC_C")) cfac = std::atof(ev) > 0 ? std::atof(ev) : cfac;
      const double c = cfac * (0.5 * kF * kF + Te);
      const double tp2d = (2.0 * kPi / L) * (2.0 * kPi / L);
      double hfac = (cs.terms & OFDFT_TERM_HARTREE) ? 1.5 : 0.0;
      if (const char* ev = std::getenv("OFDFT_PREC_H")) hfac = std::atof(ev) >= 0 ? std::atof(ev) : hfac;
      double kfac = use_na() ? 1.0 : 0.0;
      if (const char* ev = std::getenv("OFDFT_PREC_K")) kfac = std::atof(ev);
      std::vector<double> Kh;
      if (kfac != 0.0 && use_na()) {
        Kh.resize(nm2);
        OFDFT_CK(cudaMemcpyAsync(Kh.data(), Kd, nm2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        OFDFT_CK(cudaStreamSynchronize(st));
      }
      const double kcurv = 4.0 * cs.alpha * cs.alpha * std::pow(nbar, 2.0 * cs.alpha - 1.0);
      std::vector<T> ph_(nm2);
      for (int m2 = 0; m2 < nm2; ++m2) {
        const double hart = m2 > 0 ? hfac * 8.0 * kPi * nbar / (tp2d * m2) : 0.0;
        const double kk = Kh.empty() ? 0.0 : kfac * kcurv * Kh[m2];
        // (the kernel is negative at large G; h stays above c / 1000)
        ph_[m2] = (T)(c / std::max(1e-3 * c, c + 0.5 * tp2d * m2 + hart + kk));
      }
      if ((rc = alloc(&precT, nm2))) return rc;
      OFDFT_CK(cudaMemcpyAsync(precT, ph_.data(), nm2 * sizeof(T), cudaMemcpyHostToDevice, st));
      OFDFT_CK(cudaStreamSynchronize(st));
    }
    // |G|^2 range of the G-space sums that fall off as Gaussians in |G| (the
    // local pseudopotential exp(-G^2 rc^2/4), the Ewald reciprocal terms):
    // below e^-39 = 1e-17 of their G = 0 size in FP64 plans, below e^-20.8 =
    // 1e-9 in FP32 plans, each far under its precision's rounding.  V_loc,
    // E_loc, the forces' G list and the structure factor's rows use it; the
    // Ewald splitting (ewald_eta) does not depend on the precision.
    g2cut_loc = (sizeof(T) == 4 ? 4.0 * 20.8 : 4.0 * 39.0) / (cs.rc * cs.rc);
    {
      // structure-factor tables by m^2 (FP64, host): v~(G)/Omega per unit charge
      // (-4 pi exp(-G^2 rc^2/4)/G^2, pi rc^2 at G = 0) and the Ewald reciprocal
      // weight (2 pi/Omega) exp(-G^2/(4 eta^2))/G^2
      const double tp2d = (2.0 * kPi / L) * (2.0 * kPi / L);
      const double eta = ewald_eta();
      std::vector<double2> tab(nm2);
      for (int m2 = 0; m2 < nm2; ++m2) {
        const double G2 = tp2d * m2;
        if (m2 == 0) { tab[m2] = make_double2(kPi * cs.rc * cs.rc / Omega, 0.0); continue; }
        tab[m2] = make_double2(-4.0 * kPi * std::exp(-G2 * cs.rc * cs.rc / 4.0) / G2 / Omega,
                               2.0 * kPi / Omega * std::exp(-G2 / (4.0 * eta * eta)) / G2);
      }
      if ((rc = alloc(&sf_tab, nm2))) return rc;
      OFDFT_CK(cudaMemcpyAsync(sf_tab, tab.data(), nm2 * sizeof(double2), cudaMemcpyHostToDevice, st));
      OFDFT_CK(cudaStreamSynchronize(st));
    }
    {
      const double tp2 = (2.0 * kPi / L) * (2.0 * kPi / L);
      // entries per (kx, ky) row: kz = 0 .. kz_max with kz^2 <= g2cut/tp2 - mx^2 - my^2
      n_vloc = 0;
      const double lim = g2cut_loc / tp2;
      for (int kx = 0; kx < n; ++kx)
        for (int ky = 0; ky < n; ++ky) {
          const int mx = kx <= (n - 1) / 2 ? kx : kx - n, my = ky <= (n - 1) / 2 ? ky : ky - n;
          const double r = lim - (double)(mx * mx + my * my);
          if (r < 0) continue;
          int kzm = (int)std::sqrt(r);
          while (kzm + 1 < nh && (double)(kzm + 1) * (kzm + 1) <= r) ++kzm;
          while (kzm >= 0 && (double)kzm * kzm > r) --kzm;
          n_vloc += (size_t)std::min(kzm, nh - 1) + 1;
        }
    }
    OFDFT_CK(cudaStreamSynchronize(st));
    return OFDFT_OK;
  }

  long long grid_points() const override { return (long long)N; }

  // |G|^2 range of the structure factor's rows and the Ewald reciprocal sum
  double ewald_g2max() const {
    const double gnyq = kPi * n / L;
    return std::min(g2cut_loc, gnyq * gnyq);
  }
  // Ewald splitting: reciprocal weights exp(-G^2/(4 eta^2)) at e^-39 at the
  // FP64 range (or the grid's Nyquist |G|), for both precisions
  double ewald_eta() const {
    const double gnyq = kPi * n / L;
    return std::sqrt(std::min(156.0 / (cs.rc * cs.rc), gnyq * gnyq) / (4.0 * 39.0));
  }

  bool tiles_fit(int r, int j) const {
    const size_t lim = 227 * 1024;
    const size_t zf = align16((size_t)2 * r * n * sizeof(T)) + 2 * zbuf_elems(n, r, zpitch()) * sizeof(C);
    const size_t zi = zinv_bytes(r);
    const size_t yx = 3 * (size_t)n * j * sizeof(C);
    return r >= 8 && j >= 8 && (j & (j - 1)) == 0 && zf <= lim && zi <= lim && yx <= lim && j <= 64 && r <= 64;
  }

  // The dynamic shared-memory limit is a property of the kernel function, not
  // of a plan, so it is raised once to the device's opt-in maximum (it bounds
  // what a launch may request; occupancy follows what each launch asks for).
  int raise_smem_limits() {
    int dev = 0, lim = 0;
    OFDFT_CK(cudaGetDevice(&dev));
    OFDFT_CK(cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // dynamic limit = opt-in maximum minus the kernel's own static shared
    // memory; set once per (device, kernel) for the process (plan creation
    // stays cheap for the serving loop), after checking this plan's need
    static std::mutex mu;
    static std::set<std::pair<int, const void*>> done;
    auto raise = [&](const void* f, size_t need) -> int {
      std::lock_guard<std::mutex> lock(mu);
      cudaFuncAttributes fa;
      OFDFT_CK(cudaFuncGetAttributes(&fa, f));
      const int dyn = lim - (int)fa.sharedSizeBytes;
      if (dyn < (int)need) { set_error("grid too large for shared memory"); return OFDFT_ERR_INVALID; }
      if (done.count({dev, f})) return OFDFT_OK;
      OFDFT_CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
      done.insert({dev, f});
      return OFDFT_OK;
    };
    int rc;
    if ((rc = raise((const void*)k_zfwd<T>, smem_zf))) return rc;
    if ((rc = raise((const void*)k_zinv_epi<T>, smem_zi))) return rc;
    if constexpr (sizeof(T) == 4) {
      if (z256 && (rc = raise((const void*)k_zfwd256<T, 8>, z256_fwd_bytes<T>(8)))) return rc;
      if (z256 && (rc = raise((const void*)k_zfwd256<T, 16>, z256_fwd_bytes<T>(16)))) return rc;
      if (z256 && (rc = raise((const void*)k_zfwd256<T, 32>, z256_fwd_bytes<T>(32)))) return rc;
      if (z256 && (rc = raise((const void*)k_zinv256<T, 8>, smem_zi256))) return rc;
      if (z256 && (rc = raise((const void*)k_zinv256<T, 16>, smem_zi256))) return rc;
      if (z256 && (rc = raise((const void*)k_zinv256<T, 32>, smem_zi256))) return rc;
    }
    if (z256 && (rc = raise((const void*)k_ypass256<T, -1>, y256_bytes<T>()))) return rc;
    if (z256 && (rc = raise((const void*)k_ypass256<T, 1>, y256_bytes<T>()))) return rc;
    if (z256 && (rc = raise((const void*)k_xgspace256<T>, x256_bytes<T>()))) return rc;
    if constexpr (sizeof(T) == 4)
      if (p256 && (rc = raise((const void*)k_plane256cl<T>, p256_bytes<T>()))) return rc;
    if ((rc = raise((const void*)k_ypass<T, -1>, smem_y))) return rc;
    if ((rc = raise((const void*)k_ypass<T, 1>, smem_y))) return rc;
    if ((rc = raise((const void*)k_xgspace<T>, smem_x))) return rc;
    if ((rc = raise((const void*)k_xpass<T, -1>, smem_xp))) return rc;
    if (planes && (rc = raise((const void*)plane_kern, smem_pl))) return rc;
    if (prec2 && (rc = raise((const void*)prec2_kern, smem_pl2))) return rc;
    const size_t sring = StreamCfg<T>::ring_bytes(3, 17);   // largest ring any streaming launch uses
    if ((rc = raise((const void*)k_gram<T, 1, 3>, sring))) return rc;
    if ((rc = raise((const void*)k_gram<T, 2, 3>, sring))) return rc;
    if ((rc = raise((const void*)k_gram<T, 3, 3>, sring))) return rc;
    if ((rc = raise((const void*)k_gram<T, 4, 3>, sring))) return rc;
    if ((rc = raise((const void*)k_gram<T, 1, 2>, sring))) return rc;
    if ((rc = raise((const void*)k_gram<T, 2, 2>, sring))) return rc;
    if ((rc = raise((const void*)k_gram<T, 3, 2>, sring))) return rc;
    if ((rc = raise((const void*)k_gram<T, 4, 2>, sring))) return rc;
    if ((rc = raise((const void*)k_gram<T, 5, 3>, sring))) return rc;
    if ((rc = raise((const void*)k_gram<T, 5, 2>, sring))) return rc;
    if ((rc = raise((const void*)k_lincomb<T>, sring))) return rc;
    if ((rc = raise((const void*)k_accept<T>, sring))) return rc;
    return OFDFT_OK;
  }

  int apply_geometry() {
    geometry();
    return raise_smem_limits();
  }

  int set_tiles(const int* tile) override {
    if (!tiles_fit(tile[0], tile[1]) || !tiles_fit(tile[0], tile[2])) {
      set_error("tile shape does not fit in shared memory");
      return OFDFT_ERR_INVALID;
    }
    tune.zR = tile[0]; tune.yJ = tile[1]; tune.xJ = tile[2];
    return apply_geometry();
  }

  // Time a few evaluations (at the uniform density, all terms) for each
  // candidate (rows per z block, y tile width, x tile width); keep the fastest.
  int autotune(void* stream_, int* tile, double* us_per_eval) override {
    if (!ions_set) { set_error("ofdft_structure_factor must be called before ofdft_autotune"); return OFDFT_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream_;
    OFDFT_RUN("k_fill", st, (double)N * sizeof(T), k_fill<T><<<grid_vec, kThreads, 0, st>>>(psi, (T)std::sqrt(nbar), N));
    const double Q = Ne / nbar;
    std::vector<int> rows{8, 16, 32}, cols{8, 16, 32};
    if (planes) cols = {16};           // the plane pass has no column tiles
    const Tune saved = tune;
    double best = 1e300;
    int bt[3] = {0, 0, 0};
    cudaEvent_t e0, e1;
    OFDFT_CK(cudaEventCreate(&e0));
    OFDFT_CK(cudaEventCreate(&e1));
    int rc = OFDFT_OK;
    for (int r : rows) {
      if ((size_t)r > (size_t)n * n) continue;
      for (int j : cols) {
        if (!tiles_fit(r, j)) continue;
        tune.zR = r; tune.yJ = j; tune.xJ = j;
        if ((rc = apply_geometry())) break;
        const int reps = 4;
        for (int w = 0; w < 1 + reps && !rc; ++w) {
          if (w == 1) OFDFT_CK(cudaEventRecord(e0, st));
          rc = eval(1, nullptr, psi, psi, 0.0, Ne / Q, Q, Q, gp, st, false);
        }
        if (rc) break;
        OFDFT_CK(cudaEventRecord(e1, st));
        OFDFT_CK(cudaEventSynchronize(e1));
        float ms = 0;
        OFDFT_CK(cudaEventElapsedTime(&ms, e0, e1));
        const double us = 1e3 * ms / reps;
        if (us < best) { best = us; bt[0] = r; bt[1] = j; bt[2] = j; }
      }
      if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc || bt[0] == 0) {
      tune = saved;
      apply_geometry();
      return rc ? rc : OFDFT_ERR_INVALID;
    }
    tune.zR = bt[0]; tune.yJ = bt[1]; tune.xJ = bt[2];
    if ((rc = apply_geometry())) return rc;
    if (tile) { tile[0] = bt[0]; tile[1] = bt[1]; tile[2] = bt[2]; }
    if (us_per_eval) *us_per_eval = best;
    return OFDFT_OK;
  }

  // Sum columns of partials[rows][cols] into res_d[off ...] (fixed order).
  int sum_partials(int rows, int cols, int off, cudaStream_t st) {
    if (cols > 256) { set_error("sum_partials: too many columns"); return OFDFT_ERR_INVALID; }
    OFDFT_RUN("k_sum_columns", st, (double)rows * cols * 8, k_sum_columns<<<1, 256, 0, st>>>(partials, rows, cols, res_d + off));
    return OFDFT_OK;
  }

  int set_ions(const double* pos, int on_device, void* S_out, void* stream_) override {
    cudaStream_t st = (cudaStream_t)stream_;
    const int nion = (int)cs.Z.size();
    OFDFT_CK(cudaMemcpyAsync(pos_d, pos, (size_t)nion * 3 * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    const int tot = nion * 3 * n;
    OFDFT_RUN("k_phases", st, (double)tot * 16, k_phases<<<std::min(4096, (tot + 255) / 256), 256, 0, st>>>(pos_d, nion, n, L, phases));
    const double g2max = ewald_g2max();
    const double eta = ewald_eta();
    const int full = S_out != nullptr;
    // rows are also kept out to |m|^2 = 600 for the S_ei shells
    const double g2rows = std::max(g2max, (2.0 * kPi / L) * (2.0 * kPi / L) * 600.0);
    // without the full S(G), only rows with |mx|, |my| <= mlim can reach g2rows:
    // zero everything, then compute that square of rows
    int mlim = (int)std::floor(std::sqrt(g2rows) / (2.0 * kPi / L));
    if (full || mlim > (n - 1) / 2) mlim = -1;
    const int nrows = mlim < 0 ? n * n : (2 * mlim + 1) * (2 * mlim + 1);
    if (mlim >= 0) {
      OFDFT_CK(cudaMemsetAsync(Sg, 0, NH * sizeof(C), st));
      OFDFT_CK(cudaMemsetAsync(vloc, 0, NH * sizeof(C), st));
      OFDFT_CK(cudaMemsetAsync(SZg, 0, NH * sizeof(C), st));
    }
    // ions per shared-memory chunk: staged kz phases within 36 KB, so that
    // with the row phases (8 x 64 complex), the charges and the kernel's own
    // static scratch the block stays inside the default 48 KB (FP64, n = 80)
    const int sch = std::max(1, std::min(64, (int)(36864 / ((size_t)nh * sizeof(C)))));
    const size_t ssm = (size_t)sch * nh * sizeof(C) + (size_t)kStructRows * sch * sizeof(C) + (size_t)sch * sizeof(T);
    const int sgrid = (nrows + kStructRows - 1) / kStructRows;
    // one ion species (every workload here): S_Z = Z S, so the kernel sums S only
    bool uni = true;
    for (double z : cs.Z) uni = uni && z == cs.Z[0];
    if (uni) OFDFT_RUN("k_struct", st, (double)NH * sizeof(C) * (full ? 2 : 1), k_struct<T, true><<<sgrid, 32 * kStructRows, ssm, st>>>(phases, Z_d, nion, n, L, sf_tab, g2rows, full, mlim, sch, Sg, vloc, SZg, partials));
    else OFDFT_RUN("k_struct", st, (double)NH * sizeof(C) * (full ? 2 : 1), k_struct<T, false><<<sgrid, 32 * kStructRows, ssm, st>>>(phases, Z_d, nion, n, L, sf_tab, g2rows, full, mlim, sch, Sg, vloc, SZg, partials));
    int rc;
    if ((rc = sum_partials(sgrid, 1, 0, st))) return rc;
    const double rcut = 6.3 / eta;
    // images per axis around minimum-image displacements
    const int nimg_mi = (int)std::ceil(rcut / L + 0.5);
    ew_eta = eta; ew_rcut = rcut; ew_nimg = nimg_mi;
    const long ncomb = (long)nion * nion * (2 * nimg_mi + 1) * (2 * nimg_mi + 1) * (2 * nimg_mi + 1);
    const int gb = (int)std::min<long>(std::min<long>(2048, 4L * nsm), (ncomb + 255) / 256);
    OFDFT_RUN("k_ewald_real", st, (double)nion * 32, k_ewald_real<<<gb, 256, 0, st>>>(pos_d, Z_d, nion, L, eta, rcut, nimg_mi, partials));
    if ((rc = sum_partials(gb, 1, 1, st))) return rc;
    OFDFT_CK(cudaMemcpyAsync(res_h, res_d, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    OFDFT_CK(cudaStreamSynchronize(st));
    double zz = 0;
    for (double z : cs.Z) zz += z * z;
    E_ion = res_h[0] + res_h[1] - eta / std::sqrt(kPi) * zz - kPi * Ne * Ne / (2.0 * Omega * eta * eta);
    if (planes)
      OFDFT_RUN("k_vloc_planes", st, 2.0 * NH * sizeof(C), k_vloc_planes<T><<<4 * nsm, 256, 0, st>>>(vloc, vloc_pl, rev_d, n));
    if (p256_possible())
      OFDFT_RUN("k_vloc_planes256", st, 2.0 * NH * sizeof(C), k_vloc_planes256<T><<<4 * nsm, 256, 0, st>>>(vloc, vloc_pl));
    if (S_out) OFDFT_CK(cudaMemcpyAsync(S_out, Sg, NH * sizeof(C), cudaMemcpyDeviceToDevice, st));
    OFDFT_CK(cudaStreamSynchronize(st));
    ions_set = true;
    return OFDFT_OK;
  }

  // One evaluation.  mode 0: density rho; mode 1: psi + t d with scale.
  // Leaves results in res_d[0..13]; copies them to res_h when sync != 0.
  // dsc (device, optional): the trial's scale and psi shift as formed by
  // k_lincomb (TrialScale); the host values scale, Q, psid are then only used
  // when sync is set, and the caller finishes with finish_eval instead.
  int eval(int mode, const T* rho, const T* ps, const T* dd, double t, double scale, double Q, double psid,
           T* out, cudaStream_t st, bool sync, double mu_ref = 0.0, const double* dsc = nullptr) {
    Spectra<T> sp = spectra();
    // psi of the uniform density: sqrt(nbar) for a given rho, sqrt(nbar / scale) for psi + t d
    const double psi_bar = std::sqrt(nbar / (mode == 0 ? 1.0 : scale));
    ProArgs<T> pa{mode, rho, ps, dd, (T)t, (T)scale, (T)cs.alpha, (T)psi_bar, dsc};
    const double tp = 2.0 * kPi / L;
    using TV = typename TreeVal<T>::type;          // 8 bytes, like the double slots of partials
    TV* pt = reinterpret_cast<TV*>(partials);
    GArgs<T> ga{(cs.terms & OFDFT_TERM_LOC) ? ((planes || p256) ? vloc_pl : vloc) : nullptr, Kt, (T)(tp * tp), (T)Omega,
                (T)(0.5 * Omega), (T)(1.0 / (double)N), (T)g2cut_loc, (cs.terms & OFDFT_TERM_HARTREE) ? 1 : 0,
                pt};
    int g_rows = 0;                       // rows of G-space partials [g_rows][4]
    if (sp.nact > 0) {
      const double zb = (double)(mode == 0 ? 1 : 2) * N * sizeof(T) + (double)sp.nact * NH * sizeof(C);
      if (z256) {
        if (int rc = launch_zfwd256(pa, sp, zb, st)) return rc;
      } else OFDFT_RUN("k_zfwd", st, zb, k_zfwd<T><<<grid_z, kThreads, smem_zf, st>>>(pa, sp, ph, tw_h, tw_n, n, zR, zP));
      if (planes) {
        OFDFT_RUN("k_plane", st, 2.0 * sp.nact * NH * sizeof(C) + ((cs.terms & OFDFT_TERM_LOC) ? (double)n_vloc * sizeof(C) : 0.0), plane_kern<<<dim3(nh, sp.nact), kPlaneThreads, smem_pl, st>>>(sp, ga, pn, rev_d, tw_n));
        g_rows = nh * sp.nact;
      } else if (p256) {
        const double pb = 2.0 * sp.nact * NH * sizeof(C) + ((cs.terms & OFDFT_TERM_LOC) ? (double)n_vloc * sizeof(C) : 0.0);
        if (int rc = launch_p256(sp, ga, sp.nact, pb, st)) return rc;
        g_rows = P256::CL * nh * sp.nact;
      } else if (z256) {
        const double yb = 2.0 * sp.nact * NH * sizeof(C);
        const double xb = yb + ((cs.terms & OFDFT_TERM_LOC) ? (double)n_vloc * sizeof(C) : 0.0);
        OFDFT_RUN("k_ypass256", st, yb, k_ypass256<T, -1><<<dim3(kGridY256, sp.nact), kThreads, y256_bytes<T>(), st>>>(sp, tw_n));
        OFDFT_RUN("k_xgspace256", st, xb, k_xgspace256<T><<<dim3(kGridX256, sp.nact), kThreads, x256_bytes<T>(), st>>>(sp, ga, tw_n));
        OFDFT_RUN("k_ypass256", st, yb, k_ypass256<T, 1><<<dim3(kGridY256, sp.nact), kThreads, y256_bytes<T>(), st>>>(sp, tw_n));
        g_rows = kGridX256 * sp.nact;
      } else {
        OFDFT_RUN("k_ypass", st, 2.0 * sp.nact * NH * sizeof(C), k_ypass<T, -1><<<dim3(grid_y1, sp.nact), kThreads, smem_y, st>>>(sp, pn, tw_n, n, yJ));
        OFDFT_RUN("k_xgspace", st, 2.0 * sp.nact * NH * sizeof(C) + ((cs.terms & OFDFT_TERM_LOC) ? (double)n_vloc * sizeof(C) : 0.0), k_xgspace<T><<<dim3(grid_x, sp.nact), kThreads, smem_x, st>>>(sp, ga, pn, tw_n, n, xJ));
        OFDFT_RUN("k_ypass", st, 2.0 * sp.nact * NH * sizeof(C), k_ypass<T, 1><<<dim3(grid_y1, sp.nact), kThreads, smem_y, st>>>(sp, pn, tw_n, n, yJ));
        g_rows = grid_x * sp.nact;
      }
    }
    // epilogue partials after room for 3 fields of G-space rows
    TV* pe = pt + (size_t)std::max(z256 ? kGridX256 : grid_x, nh) * 3 * 4;
    if (mode == 0) mu_ref = 0.0;
    FinArgs<T> fa{pt, g_rows, pe, grid_z, res_d};
    const double cy = 9.8696044010893586188344909998762 / (1.4142135623730950488016887242097 * std::pow(Te, 1.5));
    EpiArgs<T> ea{mode, rho, ps, dd, (T)t, (T)scale, (T)cs.alpha, (T)Te, (T)cy, (T)mu_ref, cs.terms, out, pe, fa,
                  counters + 0, nullptr, nullptr, dsc, cs.fd64 ? 1 : 0, cy};
    const double eb = (double)sp.nact * NH * sizeof(C) + (double)(mode == 0 ? 1 : 2) * N * sizeof(T) + (out ? (double)N * sizeof(T) : 0.0);
    if (z256) {
      if (int rc = launch_zinv256(sp, ea, eb, st)) return rc;
    } else OFDFT_RUN("k_zinv_epi", st, eb, k_zinv_epi<T><<<grid_z, kThreads, smem_zi, st>>>(sp, ea, ph, tw_h, tw_n, n, zR, zP));
    if (sync) {
      OFDFT_CK(cudaMemcpyAsync(res_h, res_d, 12 * sizeof(double), cudaMemcpyDeviceToHost, st));
      OFDFT_CK(cudaStreamSynchronize(st));
      finish_eval(mode, scale, Q, psid, mu_ref, sp.merged != 0);
    }
    return OFDFT_OK;
  }

  // out = P in = IFFT[p(G) FFT(in)/N]: the psi-field transform chain on a
  // plain vector with the G-space factor p(m^2) (GArgs::prec, EpiArgs mode 3)
  int precondition(const T* in, T* out, cudaStream_t st, const T* pold = nullptr, T* pyout = nullptr) {
    Spectra<T> sp{};
    sp.s[2] = spec[2]; sp.nact = 1; sp.idx[0] = 2; sp.merged = 0; sp.planes = (planes || prec2 || p256) ? 1 : 0;
    ProArgs<T> pa{1, nullptr, in, nullptr, (T)0, (T)1, (T)cs.alpha, (T)0};
    const double tp = 2.0 * kPi / L;
    using TV = typename TreeVal<T>::type;
    TV* pt = reinterpret_cast<TV*>(partials);
    GArgs<T> ga{nullptr, Kt, (T)(tp * tp), (T)Omega, (T)(0.5 * Omega), (T)(1.0 / (double)N), (T)g2cut_loc, 0, pt,
                precT};
    const double fb = 2.0 * NH * sizeof(C);
    if (z256) {
      if (int rc = launch_zfwd256(pa, sp, (double)N * sizeof(T) + NH * sizeof(C), st)) return rc;
    } else OFDFT_RUN("k_zfwd", st, (double)N * sizeof(T) + NH * sizeof(C), k_zfwd<T><<<grid_z, kThreads, smem_zf, st>>>(pa, sp, ph, tw_h, tw_n, n, zR, zP));
    if (prec2) {
      // one field: two blocks (a cluster) per kz plane
      OFDFT_RUN("k_plane_prec2", st, fb, prec2_kern<<<dim3(2 * nh), kPlaneThreads, smem_pl2, st>>>(sp, ga, pn, rev_d, tw_n));
    } else if (planes) {
      OFDFT_RUN("k_plane", st, fb, plane_kern<<<dim3(nh, 1), kPlaneThreads, smem_pl, st>>>(sp, ga, pn, rev_d, tw_n));
    } else if (p256) {
      if (int rc = launch_p256(sp, ga, 1, fb, st)) return rc;
    } else if (z256) {
      OFDFT_RUN("k_ypass256", st, fb, k_ypass256<T, -1><<<dim3(kGridY256, 1), kThreads, y256_bytes<T>(), st>>>(sp, tw_n));
      OFDFT_RUN("k_xgspace256", st, fb, k_xgspace256<T><<<dim3(kGridX256, 1), kThreads, x256_bytes<T>(), st>>>(sp, ga, tw_n));
      OFDFT_RUN("k_ypass256", st, fb, k_ypass256<T, 1><<<dim3(kGridY256, 1), kThreads, y256_bytes<T>(), st>>>(sp, tw_n));
    } else {
      OFDFT_RUN("k_ypass", st, fb, k_ypass<T, -1><<<dim3(grid_y1, 1), kThreads, smem_y, st>>>(sp, pn, tw_n, n, yJ));
      OFDFT_RUN("k_xgspace", st, fb, k_xgspace<T><<<dim3(grid_x, 1), kThreads, smem_x, st>>>(sp, ga, pn, tw_n, n, xJ));
      OFDFT_RUN("k_ypass", st, fb, k_ypass<T, 1><<<dim3(grid_y1, 1), kThreads, smem_y, st>>>(sp, pn, tw_n, n, yJ));
    }
    TV* pe = pt + (size_t)std::max(z256 ? kGridX256 : grid_x, nh) * 3 * 4;
    FinArgs<T> fa{pt, 0, pe, 0, res_d};
    EpiArgs<T> ea{3, nullptr, in, in, (T)0, (T)1, (T)cs.alpha, (T)Te, (T)1, (T)0, cs.terms, out, pe, fa,
                  counters + 0, pold, pyout};
    const double pb = (double)NH * sizeof(C) + (double)N * sizeof(T) * (pyout ? 3.0 : 1.0);
    if (z256) {
      if (int rc = launch_zinv256(sp, ea, pb, st)) return rc;
    } else OFDFT_RUN("k_zinv_epi", st, pb, k_zinv_epi<T><<<grid_z, kThreads, smem_zi, st>>>(sp, ea, ph, tw_h, tw_n, n, zR, zP));
    return OFDFT_OK;
  }

  // From the 12 raw sums in res_h[0..11] (see finalize_eval) to
  // res_h: 0 F_TF 1 E_vW 2 E_NL 3 E_H 4 E_loc 5 E_xc 6 E_ion 7 F_total 8 N_e
  // 9 mu 10 residual 11 slope <g, d> 12 int v_rest n 13 nonfinite count.
  void finish_eval(int mode, double scale_t, double Q_t, double psid, double mu_ref, bool merg) {
    double s[12];
    std::memcpy(s, res_h, sizeof(s));
    const double scale = mode == 0 ? 1.0 : scale_t;
    const double E_H = s[0], E_loc = s[1], E_NL = merg ? s[2] * scale : s[2];
    const double E_vW = s[3] * scale;
    // int v_NL n = 2 a E_NL = E_NL for a = 1/2 (merged: v_NL is not in the epilogue's v_rest)
    const double F_TF = s[4] * dV, E_xc = s[5] * dV, vn = s[6] * dV + (merg ? E_NL : 0.0);
    const double gd = s[7] * dV, gg = s[8] * dV, gpsi = s[9] * dV, ne = s[10] * dV;
    const double tot = F_TF + E_vW + E_NL + E_H + E_loc + E_xc + E_ion;
    const double Nel = mode == 0 ? ne : Ne;
    const double mu = (vn + E_vW) / Nel;
    // residual^2 = (1/Q) int (g' - (mu - mu_ref) psi)^2, Q = int psi^2 (= N_e for mode 0)
    const double Q = mode == 0 ? ne : Q_t;
    const double dm = mu - mu_ref;
    const double r2 = (gg - 2.0 * dm * gpsi + dm * dm * Q) / Q;
    double* r = res_h;
    r[0] = F_TF; r[1] = E_vW; r[2] = E_NL; r[3] = E_H; r[4] = E_loc; r[5] = E_xc; r[6] = E_ion;
    r[7] = tot; r[8] = ne; r[9] = mu; r[10] = std::sqrt(std::max(r2, 0.0));
    // slope dE/dt = <g, d> with g = 2 scale (g' - (mu - mu_ref) psi_t)
    r[11] = 2.0 * scale * (gd - dm * psid);
    r[12] = vn; r[13] = s[11];
  }

  int energy_potential(const void* rho, void* v_out, ofdft_energies* e, void* stream_) override {
    if (!ions_set) { set_error("ofdft_structure_factor must be called before evaluations"); return OFDFT_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream_;
    int rc = eval(0, (const T*)rho, nullptr, nullptr, 0.0, 1.0, 0.0, 0.0, (T*)v_out, st, e != nullptr);
    if (rc) return rc;
    if (e) fill_energies(e);
    return OFDFT_OK;
  }

  int energy_potential_async(const void* rho, void* v_out, double* e_dev, void* stream_) override {
    if (!ions_set) { set_error("ofdft_structure_factor must be called before evaluations"); return OFDFT_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream_;
    int rc = eval(0, (const T*)rho, nullptr, nullptr, 0.0, 1.0, 0.0, 0.0, (T*)v_out, st, false);
    if (rc) return rc;
    OFDFT_RUN("k_finish_energies", st, 23 * 8.0, k_finish_energies<<<1, 32, 0, st>>>(res_d, dV, E_ion, merged() ? 1 : 0, e_dev));
    return OFDFT_OK;
  }

  void fill_energies(ofdft_energies* e) const {
    e->F_TF = res_h[0]; e->E_vW = res_h[1]; e->E_NL = res_h[2]; e->E_H = res_h[3];
    e->E_loc = res_h[4]; e->E_xc = res_h[5]; e->E_ion = res_h[6]; e->F_total = res_h[7];
    e->N_e = res_h[8]; e->mu = res_h[9]; e->residual = res_h[10];
  }

  // ------------------------------------------------------------------
  // dot products <V_i, W_j> for host-side use (chunks of kMaxV vectors)
  int gram(const std::vector<const T*>& V, const std::vector<const T*>& W, std::vector<double>& out,
           cudaStream_t st, bool readback = true) {
    const int nv = (int)V.size(), nw = (int)W.size();
    if ((size_t)nv * nw > 104 || nw > kMaxW) { set_error("gram: too many vectors"); return OFDFT_ERR_INVALID; }
    out.assign((size_t)nv * nw, 0.0);
    // every chunk's last block writes its columns to res_d[16 + c0 * nw ...]
    const int chunk = std::min(kMaxV, kMaxLin - nw);      // a launch streams cn + nw <= kMaxLin vectors
    for (int c0 = 0; c0 < nv; c0 += chunk) {
      const int cn = std::min(chunk, nv - c0);
      VecList<T> xl{}; xl.nv = cn + nw;
      for (int i = 0; i < cn; ++i) xl.v[i] = V[c0 + i];
      for (int j = 0; j < nw; ++j) xl.v[cn + j] = W[j];
      double* o = res_d + 16 + (size_t)c0 * nw;
      const int S = cn + nw <= 17 ? 3 : 2;   // k_gram is built for 2 or 3 ring stages
      const size_t sm = std::max(StreamCfg<T>::ring_bytes(S, cn + nw), tree_scratch_bytes<T>(cn * nw, kStreamThreads));
      prof.begin("k_gram", st, (double)(cn + nw) * N * sizeof(T));
      auto launch = [&](auto kern) { kern<<<grid_stream, kStreamThreads, sm, st>>>(xl, cn, Nv, partials, counters + 1, o); };
      switch (nw * 8 + S) {
        case 1 * 8 + 3: launch(k_gram<T, 1, 3>); break;
        case 2 * 8 + 3: launch(k_gram<T, 2, 3>); break;
        case 3 * 8 + 3: launch(k_gram<T, 3, 3>); break;
        case 4 * 8 + 3: launch(k_gram<T, 4, 3>); break;
        case 5 * 8 + 3: launch(k_gram<T, 5, 3>); break;
        case 1 * 8 + 2: launch(k_gram<T, 1, 2>); break;
        case 2 * 8 + 2: launch(k_gram<T, 2, 2>); break;
        case 3 * 8 + 2: launch(k_gram<T, 3, 2>); break;
        case 4 * 8 + 2: launch(k_gram<T, 4, 2>); break;
        case 5 * 8 + 2: launch(k_gram<T, 5, 2>); break;
        default: set_error("gram: no kernel for this list"); return OFDFT_ERR_INVALID;
      }
      prof.end(st);
      OFDFT_LAUNCH_CK();
    }
    if (!readback) return OFDFT_OK;
    int rc;
    if ((rc = read_results(st))) return rc;
    for (int i = 0; i < nv; ++i)
      for (int j = 0; j < nw; ++j) out[(size_t)i * nw + j] = res_h[16 + i * nw + j] * dV;
    return OFDFT_OK;
  }

  // out = sum_i c_i V_i; returns <out,out>, <out,g>, <out,psi> (times dV);
  // with dd == nullptr the dots are not read back (no host synchronisation)
  int lincomb(const VecList<T>& terms, T* out, double* dd, double* dg, double* dpsi, cudaStream_t st,
              TrialScale ts = TrialScale{}, const double* dcoef = nullptr) {
    VecList<T> xl = terms;
    const int nv = terms.nv;
    xl.v[nv] = g; xl.v[nv + 1] = psi;
    xl.nv = nv + 2;
    OFDFT_RUN("k_lincomb", st, (double)(nv + 3) * N * sizeof(T),
              k_lincomb<T><<<grid_stream, kStreamThreads, StreamCfg<T>::ring_bytes(stream_stages(kMaxLin - 1), nv + 2), st>>>(
                  xl, nv, out, Nv, partials, counters + 2, res_d + 16, ts, dcoef));
    if (!dd) return OFDFT_OK;
    int rc;
    if ((rc = read_results(st))) return rc;
    *dd = res_h[16] * dV; *dg = res_h[17] * dV; *dpsi = res_h[18] * dV;
    return OFDFT_OK;
  }

  // copy the reduction results res_d[16, 120) to the host
  int read_results(cudaStream_t st) {
    OFDFT_CK(cudaMemcpyAsync(res_h + 16, res_d + 16, (120 - 16) * sizeof(double), cudaMemcpyDeviceToHost, st));
    OFDFT_CK(cudaStreamSynchronize(st));
    return OFDFT_OK;
  }

  int minimize(void* rho_io, int start_uniform, const ofdft_min_opts& o, ofdft_result* r, void* stream_) override;

  int sei_shells(const void* rho, int n_shells, double* q_out, double* s_out, void* stream_) override;
  int forces(const void* rho, double* f_out_h, void* stream_) override;
  int pressure(const void* rho, double* p_out_h, void* stream_) override;
  int build_pressure_table(cudaStream_t st);
  int build_shells(int n_shells, cudaStream_t st);
  int shell_sums(const void* rho, cudaStream_t st, std::vector<double>& hout);
  int md_run(void* rho_io, int start_uniform, double* pos_io, double* vel_io, const double* mass,
             const ofdft_md_opts& o, ofdft_md_thermostat* th, int n_steps, ofdft_md_frame* frames,
             double* q_out, double* sei_sum, double* sii_sum, void* stream_) override;
};

// ---------------------------------------------------------------------------
// Strong-Wolfe line search (sufficient decrease c1, curvature c2; cubic
// interpolation in the zoom phase).  phi(t, &f, &slope) evaluates.
struct LSPoint { double t, f, g; };

static double cubic_min(const LSPoint& a, const LSPoint& b, bool* ok) {
  const double d1 = a.g + b.g - 3.0 * (a.f - b.f) / (a.t - b.t);
  const double disc = d1 * d1 - a.g * b.g;
  if (disc < 0) { *ok = false; return 0; }
  const double d2 = std::copysign(std::sqrt(disc), b.t - a.t);
  const double den = b.g - a.g + 2.0 * d2;
  if (den == 0) { *ok = false; return 0; }
  *ok = true;
  return b.t - (b.t - a.t) * (b.g + d2 - d1) / den;
}

// rel_noise: relative size of rounding noise in the energy; a trial whose
// energy change is inside it is judged on the slope alone (approximate Wolfe).
template <typename F>
static int line_search(F&& phi, double f0, double g0, double t0, double c1, double c2, int max_evals,
                       double rel_noise, LSPoint* acc, int* evals) {
  const double eps_f = rel_noise * std::max(1.0, std::fabs(f0));
  auto armijo = [&](double t, double f) { return f <= f0 + c1 * t * g0 || std::fabs(f - f0) <= eps_f; };
  auto curv = [&](double g) { return std::fabs(g) <= -c2 * g0; };
  LSPoint prev{0.0, f0, g0}, lo{}, hi{};
  double t = t0;
  *evals = 0;
  bool bracket = false;
  while (*evals < max_evals) {
    LSPoint p{t, 0, 0};
    int rc = phi(t, &p.f, &p.g);
    if (rc) return rc;
    ++*evals;
    if (!std::isfinite(p.f) || !std::isfinite(p.g)) { lo = prev; hi = p; hi.f = INFINITY; bracket = true; break; }
    if (!armijo(t, p.f) || (*evals > 1 && p.f >= prev.f && std::fabs(p.f - prev.f) > eps_f)) {
      lo = prev; hi = p; bracket = true; break;
    }
    if (curv(p.g)) { *acc = p; return OFDFT_OK; }
    if (p.g >= 0) { lo = p; hi = prev; bracket = true; break; }
    prev = p;
    t *= 2.0;
  }
  if (!bracket) return OFDFT_ERR_NOT_CONVERGED;
  while (*evals < max_evals) {
    bool ok = false;
    double tc = 0;
    if (std::isfinite(hi.f)) tc = cubic_min(lo, hi, &ok);
    const double left = std::min(lo.t, hi.t), right = std::max(lo.t, hi.t), w = right - left;
    if (!ok || !(tc >= left + 0.1 * w && tc <= right - 0.1 * w)) tc = 0.5 * (lo.t + hi.t);
    LSPoint p{tc, 0, 0};
    int rc = phi(tc, &p.f, &p.g);
    if (rc) return rc;
    ++*evals;
    if (!std::isfinite(p.f) || !armijo(tc, p.f) || (p.f >= lo.f && std::fabs(p.f - lo.f) > eps_f)) {
      hi = p;
      if (!std::isfinite(p.f)) hi.f = INFINITY;
    } else {
      if (curv(p.g)) { *acc = p; return OFDFT_OK; }
      if (p.g * (hi.t - lo.t) >= 0) hi = lo;
      lo = p;
    }
    if (std::fabs(hi.t - lo.t) < 1e-16 * std::max(1.0, std::fabs(lo.t))) break;
  }
  return OFDFT_ERR_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------
// L-BFGS on psi with n = N_e psi^2 / Q.  The two-loop recursion is carried
// out on scalars from the Gram matrices of the history; the direction is
// then one linear-combination pass.
template <typename T>
int Engine<T>::minimize(void* rho_io, int start_uniform, const ofdft_min_opts& o, ofdft_result* r, void* stream_) {
  if (!ions_set) { set_error("ofdft_structure_factor must be called before ofdft_minimize"); return OFDFT_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream_;
  const int m = std::min(o.m, m_max);
  if (m < 1) { set_error("L-BFGS memory must be >= 1"); return OFDFT_ERR_INVALID; }
  const double n_ion = (double)cs.Z.size();
  const char* trace_env = std::getenv("OFDFT_TRACE");
  const bool trace = trace_env && trace_env[0] == '1';
  int rc;
  if (start_uniform) OFDFT_RUN("k_fill", st, (double)N * sizeof(T), k_fill<T><<<grid_vec, kThreads, 0, st>>>(psi, (T)std::sqrt(nbar), N));
  else OFDFT_RUN("k_sqrt_clamp", st, 2.0 * N * sizeof(T), k_sqrt_clamp<T><<<grid_vec, kThreads, 0, st>>>(psi, (const T*)rho_io, N));
  std::vector<double> dots;
  if ((rc = gram({psi}, {psi}, dots, st))) return rc;
  double Qcur = dots[0];
  if (!(Qcur > 0)) { set_error("initial density has zero norm"); return OFDFT_ERR_INVALID; }
  int evals = 0;
  // evaluation at the starting point (t = 0; d is unused, psi stands in)
  if ((rc = eval(1, nullptr, psi, psi, 0.0, Ne / Qcur, Qcur, Qcur, gp, st, true))) return rc;
  ++evals;
  double F = res_h[7];
  double energies[14];
  std::memcpy(energies, res_h, sizeof(energies));
  if (!std::isfinite(F) || res_h[13] > 0) { set_error("non-finite energy at the starting density"); return OFDFT_ERR_NAN; }
  OFDFT_RUN("k_project", st, 3.0 * N * sizeof(T), k_project<T><<<grid_vec, kThreads, 0, st>>>(g, gp, psi, Ne / Qcur, res_h[9], N));
  double mu_ref = res_h[9];   // reference chemical potential for g' (mu of the last accepted point)

  // P g of the current g (pgv[pcur]); the previous one is kept until the next
  // preconditioning pass has formed P y = P g_new - P g_old
  int pcur = 0;
  if ((rc = precondition(g, pgv[pcur], st))) return rc;

  Ring ring; ring.m = m;
  double gg = 0;
  {
    std::vector<double> d0;
    if ((rc = gram({g, psi}, {g, psi}, d0, st))) return rc;
    gg = d0[0];
    Qcur = d0[3];
  }
  int new_slot = -1;
  int small = 0, it = 0;
  bool converged = false;
  for (it = 1; it <= o.max_iter; ++it) {
    double dd = 0, dg = 0, dpsi = 0, gamma = 1.0, t0 = 1.0;
    // with history the direction is formed from device scalars and its first
    // trial is launched right behind it; the host reads the direction's dots,
    // the trial's result and the recursion's outcome in one round trip
    bool first_ready = false;
    double first_t = 0, first_f = 0, first_slope = 0, first_E[14], first_scale = 0, first_mu = 0;
    // d = -P g (restart or first iteration); t0 = 10% of |psi| along it
    auto steepest = [&]() -> int {
      VecList<T> vl{};
      vl.nv = 1;
      vl.v[0] = pgv[pcur]; vl.c[0] = -1.0;
      int e;
      if ((e = lincomb(vl, d, &dd, &dg, &dpsi, st))) return e;
      t0 = 0.1 * std::sqrt(Qcur / std::max(dd, 1e-300));
      gamma = 1.0;
      return OFDFT_OK;
    };
    if (new_slot >= 0) {
      // P g of the new gradient, and P y_new = P g_new - P g_old on the way
      const int pnew = 1 - pcur;
      if ((rc = precondition(g, pgv[pnew], st, pgv[pcur], PYh[new_slot]))) return rc;
      pcur = pnew;
      // the accepted pair's own dots came from k_accept (res 120..125); one
      // pass dots [older s, older y, y_new] with [g, P g, y_new, P y_new]
      TwoLoopArgs ta{};
      ta.count = ring.count; ta.new_slot = new_slot; ta.dv = dV;
      std::vector<const T*> V;
      for (int i = 0; i < ring.count; ++i) {
        ta.ring_slot[i] = ring.slot(i);
        if (ring.slot(i) != new_slot) ta.old_slot[ta.no++] = ring.slot(i);
      }
      for (int i = 0; i < ta.no; ++i) V.push_back(Sh[ta.old_slot[i]]);
      for (int i = 0; i < ta.no; ++i) V.push_back(Yh[ta.old_slot[i]]);
      V.push_back(Yh[new_slot]);
      std::vector<double> cross;
      if ((rc = gram(V, {g, pgv[pcur], Yh[new_slot], PYh[new_slot]}, cross, st, false))) return rc;
      // two-loop recursion on the device (k_twoloop), then the direction
      // d = coef[0] P g + sum (coef[1+2j] P y_j + coef[2+2j] s_j)
      OFDFT_RUN("k_twoloop", st, 0.0, k_twoloop<<<1, 32, 0, st>>>(ta, res_d + 16, res_d + 120, tl_state, res_d + 129));
      VecList<T> vl{};
      vl.nv = 0;
      vl.v[vl.nv++] = pgv[pcur];
      for (int j = 0; j < ring.count; ++j) {
        vl.v[vl.nv++] = PYh[ring.slot(j)];
        vl.v[vl.nv++] = Sh[ring.slot(j)];
      }
      TrialScale ts{0.0, 1.0, Ne, dV, nbar, res_d + 126, &tl_state->Q, &tl_state->kk};
      if ((rc = lincomb(vl, d, nullptr, nullptr, nullptr, st, ts, tl_state->coef))) return rc;
      if ((rc = eval(1, nullptr, psi, d, 1.0, 1.0, 0.0, 0.0, gp, st, false, mu_ref, res_d + 126))) return rc;
      ++evals;
      OFDFT_CK(cudaMemcpyAsync(res_h, res_d, 12 * sizeof(double), cudaMemcpyDeviceToHost, st));
      OFDFT_CK(cudaMemcpyAsync(res_h + 16, res_d + 16, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
      OFDFT_CK(cudaMemcpyAsync(res_h + 126, res_d + 126, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
      OFDFT_CK(cudaStreamSynchronize(st));
      // k_accept's dots (copied after the accept) are on the host now
      Qcur = res_h[122] * dV;
      gg = res_h[123] * dV;
      gamma = res_h[129];
      if (res_h[130] == 0.0) ring.clear();   // curvature lost to rounding: history dropped
      new_slot = -1;
      dd = res_h[16] * dV; dg = res_h[17] * dV; dpsi = res_h[18] * dV;
      t0 = res_h[128];
      const double sc = res_h[126];
      finish_eval(1, sc, Qcur + 2.0 * t0 * dpsi + t0 * t0 * dd, dpsi + t0 * dd, mu_ref, merged());
      first_t = t0;
      first_f = res_h[13] > 0 ? NAN : res_h[7];
      first_slope = res_h[11];
      first_scale = sc; first_mu = res_h[9];
      std::memcpy(first_E, res_h, sizeof(first_E));
      first_ready = true;
    } else {
      if ((rc = steepest())) return rc;
    }
    if (!(dg < 0) && ring.count > 0) {
      first_ready = false;
      // not a descent direction: drop the history and restart along -P g
      ring.clear();
      if ((rc = steepest())) return rc;
    }
    if (!(dg < 0)) break;
    // --- strong-Wolfe line search along d
    double lastScale = 0, lastMu = 0, lastE[14];
    auto phi = [&](double t, double* f, double* slope) -> int {
      if (first_ready && t == first_t) {
        first_ready = false;
        *f = first_f; *slope = first_slope;
        lastScale = first_scale; lastMu = first_mu;
        std::memcpy(lastE, first_E, sizeof(lastE));
        return OFDFT_OK;
      }
      first_ready = false;
      const double Qt = Qcur + 2.0 * t * dpsi + t * t * dd;
      const double sc = Ne / Qt;
      int e = eval(1, nullptr, psi, d, t, sc, Qt, dpsi + t * dd, gp, st, true, mu_ref);
      if (e) return e;
      ++evals;
      *f = res_h[13] > 0 ? NAN : res_h[7];
      *slope = res_h[11];
      lastScale = sc; lastMu = res_h[9];
      std::memcpy(lastE, res_h, sizeof(lastE));
      return OFDFT_OK;
    };
    LSPoint acc{};
    int lsev = 0;
    // energy noise: FP64 rounding, or FP32 terms summed in FP64
    const double rel_noise = sizeof(T) == 4 ? 3e-7 : 1e-14;
    rc = line_search(phi, F, dg, t0, o.c1, o.c2, 40, rel_noise, &acc, &lsev);
    if (rc == OFDFT_ERR_NOT_CONVERGED && ring.count > 0) {
      // failed along the quasi-Newton direction: drop the history and retry once
      // along -P g (scaled as a first step) before giving up
      ring.clear();
      first_ready = false;
      if ((rc = steepest())) return rc;
      if (dg < 0) {
        int lsev2 = 0;
        rc = line_search(phi, F, dg, t0, o.c1, o.c2, 40, rel_noise, &acc, &lsev2);
        lsev += lsev2;
      }
    }
    if (trace)
      std::fprintf(stderr, "ofdft it %4d F %.12f dphi0 %.3e t %.3e ls_evals %d status %d R %.3e hist %d"
                   " gamma %.9e dd %.9e dpsi %.9e Q %.12e gg %.9e\n", it,
                   rc == OFDFT_OK ? acc.f : F, dg, acc.t, lsev, rc, lastE[10], ring.count, gamma, dd, dpsi, Qcur, gg);
    if (rc == OFDFT_ERR_NOT_CONVERGED) break;
    if (rc) return rc;
    // --- accept: s = t d, y = g_t - g, psi += t d, g = g_t  (the last trial is the accepted one)
    const int slot = ring.push();
    VecList<T> xa{};
    xa.nv = 4; xa.v[0] = psi; xa.v[1] = d; xa.v[2] = gp; xa.v[3] = g;
    OFDFT_RUN("k_accept", st, 8.0 * N * sizeof(T),
              k_accept<T><<<grid_stream, kStreamThreads, StreamCfg<T>::ring_bytes(stream_stages(4), 4), st>>>(
                  xa, (T)acc.t, (T)(2.0 * lastScale), (T)(lastMu - mu_ref), psi, g, Sh[slot], Yh[slot], Nv,
                  partials, counters + 3, res_d + 120));
    OFDFT_CK(cudaMemcpyAsync(res_h + 120, res_d + 120, 6 * sizeof(double), cudaMemcpyDeviceToHost, st));
    new_slot = slot;
    mu_ref = lastMu;
    const double dF = std::fabs(acc.f - F) / n_ion;
    F = acc.f;
    std::memcpy(energies, lastE, sizeof(energies));
    small = dF < o.tol_F_per_ion ? small + 1 : 0;
    if (small >= 3 && lastE[10] < o.tol_residual) { converged = true; break; }
  }
  // output density n = N_e psi^2 / int psi^2
  std::vector<double> qd;
  if ((rc = gram({psi}, {psi}, qd, st))) return rc;
  OFDFT_RUN("k_density", st, 2.0 * N * sizeof(T), k_density<T><<<grid_vec, kThreads, 0, st>>>((T*)rho_io, psi, Ne / qd[0], N));
  OFDFT_CK(cudaStreamSynchronize(st));
  const int status = converged ? OFDFT_OK : OFDFT_ERR_NOT_CONVERGED;
  if (r) {
    std::memcpy(res_h, energies, sizeof(energies));
    fill_energies(&r->e);
    r->iterations = std::min(it, o.max_iter);
    r->evaluations = evals;
    r->status = status;
  }
  if (!converged) set_error("minimiser stopped before reaching the tolerances");
  return status;
}


// ---------------------------------------------------------------------------
// Structure factors on |q| shells.  Shell lists for the first n_shells
// distinct nonzero m^2 on the grid.
template <typename T>
int Engine<T>::build_shells(int n_shells, cudaStream_t st) {
  if (n_shells < 1 || n_shells > 4096) { set_error("n_shells must be in [1, 4096]"); return OFDFT_ERR_INVALID; }
  if (sh_ns == n_shells) return OFDFT_OK;
  // distinct nonzero m^2 present on the grid, ascending, and their entries
  // signed wave numbers on the grid: -(n/2) .. (n-1)/2 per axis; kz = 0 .. n/2
  const int lim = n / 2, mhi = (n - 1) / 2;
  std::vector<char> present(3 * lim * lim + 1, 0);
  for (int mx = -lim; mx <= mhi; ++mx)
    for (int my = -lim; my <= mhi; ++my)
      for (int mz = 0; mz <= lim; ++mz) {
        const int m2 = mx * mx + my * my + mz * mz;
        if (m2 > 0) present[m2] = 1;
      }
  std::vector<int> shell_m2;
  for (int m2 = 1; m2 < (int)present.size() && (int)shell_m2.size() < n_shells; ++m2)
    if (present[m2]) shell_m2.push_back(m2);
  const int ns = (int)shell_m2.size();
  if (ns < n_shells) { set_error("grid has fewer distinct shells than requested"); return OFDFT_ERR_INVALID; }
  const int m2max = shell_m2.back();
  if ((2.0 * kPi / L) * (2.0 * kPi / L) * m2max > std::max(g2cut_loc, (2.0 * kPi / L) * (2.0 * kPi / L) * 600.0)) {
    set_error("requested shells extend beyond the stored structure factor");
    return OFDFT_ERR_INVALID;
  }
  std::vector<int> shell_of(m2max + 1, -1);
  for (int i = 0; i < ns; ++i) shell_of[shell_m2[i]] = i;
  std::vector<std::vector<long long>> lists(ns);
  std::vector<std::vector<float>> wl(ns);
  const int r = (int)std::ceil(std::sqrt((double)m2max));
  for (int mx = -std::min(r, lim); mx <= std::min(r, mhi); ++mx)
    for (int my = -std::min(r, lim); my <= std::min(r, mhi); ++my)
      for (int mz = 0; mz <= std::min(r, lim); ++mz) {
        const int m2 = mx * mx + my * my + mz * mz;
        if (m2 == 0 || m2 > m2max || shell_of[m2] < 0) continue;
        const int kx = mx < 0 ? mx + n : mx, ky = my < 0 ? my + n : my;
        const long long q = ((long long)kx * n + ky) * nh + mz;
        lists[shell_of[m2]].push_back(q);
        wl[shell_of[m2]].push_back((mz == 0 || 2 * mz == n) ? 1.0f : 2.0f);
      }
  std::vector<int> ptr(ns + 1, 0);
  std::vector<long long> idx;
  std::vector<float> wts;
  for (int i = 0; i < ns; ++i) {
    ptr[i + 1] = ptr[i] + (int)lists[i].size();
    idx.insert(idx.end(), lists[i].begin(), lists[i].end());
    wts.insert(wts.end(), wl[i].begin(), wl[i].end());
  }
  OFDFT_CK(cudaStreamSynchronize(st));
  free_shells();
  sh_bytes[0] = ptr.size() * sizeof(int);
  sh_bytes[1] = std::max<size_t>(1, idx.size()) * sizeof(long long);
  sh_bytes[2] = std::max<size_t>(1, wts.size()) * sizeof(float);
  sh_bytes[3] = 3 * (size_t)ns * sizeof(double);
  OFDFT_CK(cached_dev_alloc((void**)&sh_ptr, sh_bytes[0]));
  OFDFT_CK(cached_dev_alloc((void**)&sh_idx, sh_bytes[1]));
  OFDFT_CK(cached_dev_alloc((void**)&sh_w, sh_bytes[2]));
  OFDFT_CK(cached_dev_alloc((void**)&sh_out, sh_bytes[3]));
  OFDFT_CK(cudaMemcpyAsync(sh_ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  OFDFT_CK(cudaMemcpyAsync(sh_idx, idx.data(), idx.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
  OFDFT_CK(cudaMemcpyAsync(sh_w, wts.data(), wts.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  OFDFT_CK(cudaStreamSynchronize(st));
  sh_m2 = shell_m2;
  sh_ns = ns;
  sh_entries = (long long)idx.size();
  return OFDFT_OK;
}

// Per-shell sums at density rho for the cached shells: hout[3 s .. 3 s + 2] =
// (sum w Re[n_e S*] / sqrt(N_e N_i), sum w |S|^2, sum w).
template <typename T>
int Engine<T>::shell_sums(const void* rho, cudaStream_t st, std::vector<double>& hout) {
  // forward transform of rho into spec[0]
  Spectra<T> sp{};
  sp.s[0] = spec[0]; sp.nact = 1; sp.idx[0] = 0;
  ProArgs<T> pa{0, (const T*)rho, nullptr, nullptr, (T)0, (T)1, (T)cs.alpha};
  OFDFT_RUN("k_zfwd", st, (double)N * sizeof(T) + (double)NH * sizeof(C), k_zfwd<T><<<grid_z, kThreads, smem_zf, st>>>(pa, sp, ph, tw_h, tw_n, n, zR, zP));
  OFDFT_RUN("k_ypass", st, 2.0 * NH * sizeof(C), k_ypass<T, -1><<<dim3(grid_y1, 1), kThreads, smem_y, st>>>(sp, pn, tw_n, n, yJ));
  OFDFT_RUN("k_xpass", st, 2.0 * NH * sizeof(C), k_xpass<T, -1><<<dim3(grid_x, 1), kThreads, smem_xp, st>>>(sp, pn, tw_n, n, xJ));
  const double nion = (double)cs.Z.size();
  const double scale = Omega / (double)N / std::sqrt(Ne * nion);
  OFDFT_RUN("k_sei_shells", st, (double)sh_entries * (2 * sizeof(C) + 12), k_sei_shells<T><<<sh_ns, 256, 0, st>>>(spec[0], Sg, sh_ptr, sh_idx, sh_w, scale, sh_out));
  hout.resize(3 * (size_t)sh_ns);
  OFDFT_CK(cudaMemcpyAsync(hout.data(), sh_out, hout.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  OFDFT_CK(cudaStreamSynchronize(st));
  return OFDFT_OK;
}

template <typename T>
int Engine<T>::sei_shells(const void* rho, int n_shells, double* q_out, double* s_out, void* stream_) {
  if (!ions_set) { set_error("ofdft_structure_factor must be called before ofdft_sei_shells"); return OFDFT_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream_;
  int rc;
  if ((rc = build_shells(n_shells, st))) return rc;
  std::vector<double> hout;
  if ((rc = shell_sums(rho, st, hout))) return rc;
  for (int i = 0; i < sh_ns; ++i) {
    q_out[i] = 2.0 * kPi / L * std::sqrt((double)sh_m2[i]);
    s_out[i] = hout[3 * i] / hout[3 * i + 2];
  }
  return OFDFT_OK;
}

// Hellmann-Feynman forces on the ions at density rho (Methods: the forces that
// drive the molecular dynamics; at fixed n only E_loc and the Ewald energy
// depend on the ion positions).  f_out_h: host double[n_ion * 3].
template <typename T>
int Engine<T>::forces(const void* rho, double* f_out_h, void* stream_) {
  if (!ions_set) { set_error("ofdft_structure_factor must be called before ofdft_forces"); return OFDFT_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream_;
  const int nion = (int)cs.Z.size();
  const double tp = 2.0 * kPi / L;
  int rc;
  if (f_ng < 0) {
    // the G list of the local and reciprocal Ewald sums (independent of the ions)
    std::vector<int4> gl;
    std::vector<double2> gf;
    const int r = (int)std::ceil(std::sqrt(g2cut_loc) / tp);
    const bool loc = (cs.terms & OFDFT_TERM_LOC) != 0;
    for (int mx = std::max(-h, -r); mx <= std::min((n - 1) / 2, r); ++mx)
      for (int my = std::max(-h, -r); my <= std::min((n - 1) / 2, r); ++my)
        for (int kz = 0; kz <= std::min(h, r); ++kz) {
          const int m2 = mx * mx + my * my + kz * kz;
          const double G2 = tp * tp * (double)m2;
          if (m2 == 0 || G2 > g2cut_loc) continue;
          const int kx = mx < 0 ? mx + n : mx, ky = my < 0 ? my + n : my;
          const int w = (kz == 0 || 2 * kz == n) ? 1 : 2;
          gl.push_back(make_int4(kx, ky, kz, w));
          const double vfac = loc ? -4.0 * kPi * std::exp(-G2 * cs.rc * cs.rc / 4.0) / G2 : 0.0;
          const double efac = 4.0 * kPi / Omega * std::exp(-G2 / (4.0 * ew_eta * ew_eta)) / G2;
          gf.push_back(make_double2(vfac, efac));
        }
    const size_t ng = std::max<size_t>(1, gl.size());
    if ((rc = alloc(&f_gl, ng)) || (rc = alloc(&f_gf, ng)) || (rc = alloc(&f_qq, ng)) ||
        (rc = alloc(&f_pt, (size_t)nion * 3 * n)) || (rc = alloc(&f_out, (size_t)nion * 3)))
      return rc;
    if (!gl.empty()) {
      OFDFT_CK(cudaMemcpyAsync(f_gl, gl.data(), gl.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
      OFDFT_CK(cudaMemcpyAsync(f_gf, gf.data(), gf.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    }
    OFDFT_CK(cudaStreamSynchronize(st));
    f_ng = (int)gl.size();
  }
  // n~ (unnormalised) into spec[0], tiled layout
  Spectra<T> sp{};
  sp.s[0] = spec[0]; sp.nact = 1; sp.idx[0] = 0;
  ProArgs<T> pa{0, (const T*)rho, nullptr, nullptr, (T)0, (T)1, (T)cs.alpha};
  OFDFT_RUN("k_zfwd", st, (double)N * sizeof(T) + (double)NH * sizeof(C), k_zfwd<T><<<grid_z, kThreads, smem_zf, st>>>(pa, sp, ph, tw_h, tw_n, n, zR, zP));
  OFDFT_RUN("k_ypass", st, 2.0 * NH * sizeof(C), k_ypass<T, -1><<<dim3(grid_y1, 1), kThreads, smem_y, st>>>(sp, pn, tw_n, n, yJ));
  OFDFT_RUN("k_xpass", st, 2.0 * NH * sizeof(C), k_xpass<T, -1><<<dim3(grid_x, 1), kThreads, smem_xp, st>>>(sp, pn, tw_n, n, xJ));
  const int tot = nion * 3 * n;
  OFDFT_RUN("k_phases_t", st, (double)tot * (16 + sizeof(C)), k_phases_t<T><<<std::min(4096, (tot + 255) / 256), 256, 0, st>>>(phases, f_pt, tot));
  if (f_ng > 0) {
    const int gq = std::min(4 * nsm, (f_ng + 127) / 128);
    OFDFT_RUN("k_forces_q", st, (double)f_ng * (3 * sizeof(C) + 32), k_forces_q<T><<<gq, 128, 0, st>>>(spec[0], f_gl, f_gf, f_ng, SZg, n, 1.0 / (double)N, f_qq));
    OFDFT_RUN("k_forces_g", st, (double)nion * f_ng * (sizeof(C) + 16), k_forces_g<T><<<nion, 256, 0, st>>>(f_qq, f_gl, f_ng, f_pt, Z_d, n, tp, f_out));
  } else {
    OFDFT_CK(cudaMemsetAsync(f_out, 0, (size_t)nion * 3 * sizeof(double), st));
  }
  // several blocks per ion (about 4 per SM in all), shares added in a fixed order
  int nsplit = std::max(1, std::min(64, (4 * nsm + nion - 1) / nion));
  while (nsplit > 1 && (size_t)nion * nsplit * 3 > partials_cap) --nsplit;
  if ((size_t)nion * nsplit * 3 > partials_cap) { set_error("forces: too many ions for the scratch"); return OFDFT_ERR_INVALID; }
  OFDFT_RUN("k_ewald_force_real", st, (double)nion * nion * 32, k_ewald_force_real<<<nion * nsplit, 256, 0, st>>>(pos_d, Z_d, nion, L, ew_eta, ew_rcut, ew_nimg, nsplit, partials));
  OFDFT_RUN("k_sum_force_parts", st, (double)nion * nsplit * 24, k_sum_force_parts<<<(3 * nion + 127) / 128, 128, 0, st>>>(partials, nion, nsplit, f_out));
  OFDFT_CK(cudaMemcpyAsync(f_out_h, f_out, (size_t)nion * 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  OFDFT_CK(cudaStreamSynchronize(st));
  return OFDFT_OK;
}

// pnl(m^2) = (3 - 6a) K(m^2) + dK/dlambda, dK the derivative of the kernel
// K(|G|/lambda; nbar/lambda^3) along the dilation at lambda = 1: Richardson
// extrapolation of central differences with steps 2e-3 and 1e-3 (the kernel is
// a Lindhard quadrature with no closed form; error O(step^4)).
template <typename T>
int Engine<T>::build_pressure_table(cudaStream_t st) {
  const int nm2 = 3 * h * h + 1;
  int rc;
  if (!p_tab && (rc = alloc(&p_tab, (size_t)5 * nm2 + 16))) return rc;
  const double lam[4] = {1.002, 0.998, 1.001, 0.999};
  double* mp = p_tab + (size_t)5 * nm2;
  for (int i = 0; i < 4; ++i) {
    const double nb = nbar / (lam[i] * lam[i] * lam[i]);
    const double y = 9.8696044010893586188 * nb / (1.4142135623730950488 * std::pow(Te, 1.5));
    OFDFT_RUN("k_mean_density", st, 32.0, k_mean_density<<<1, kMeanThreads, 0, st>>>(y, Te, mp + 4 * i));
  }
  std::vector<double> mph(16);
  OFDFT_CK(cudaMemcpyAsync(mph.data(), mp, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
  OFDFT_CK(cudaStreamSynchronize(st));
  for (int i = 0; i < 4; ++i) {
    KernArgs ka{L * lam[i], nbar / (lam[i] * lam[i] * lam[i]), Te, mph[4 * i + 1], mph[4 * i + 2], cs.alpha, nm2};
    OFDFT_RUN("k_kernel_table", st, (double)nm2 * 8, k_kernel_table<<<kernel_table_blocks(nm2), 32 * kKernWarps, 0, st>>>(ka, p_tab + (size_t)i * nm2));
  }
  std::vector<double> tabs((size_t)4 * nm2), K0(nm2), pnl(nm2);
  OFDFT_CK(cudaMemcpyAsync(tabs.data(), p_tab, tabs.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  OFDFT_CK(cudaMemcpyAsync(K0.data(), Kd, nm2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  OFDFT_CK(cudaStreamSynchronize(st));
  for (int m = 0; m < nm2; ++m) {
    const double c1 = (tabs[m] - tabs[(size_t)nm2 + m]) / (2.0 * 2e-3);
    const double c2 = (tabs[(size_t)2 * nm2 + m] - tabs[(size_t)3 * nm2 + m]) / (2.0 * 1e-3);
    pnl[m] = (3.0 - 6.0 * cs.alpha) * K0[m] + (4.0 * c2 - c1) / 3.0;
  }
  OFDFT_CK(cudaMemcpyAsync(p_tab + (size_t)4 * nm2, pnl.data(), nm2 * sizeof(double), cudaMemcpyHostToDevice, st));
  OFDFT_CK(cudaStreamSynchronize(st));
  p_ready = true;
  return OFDFT_OK;
}

// Pressure P = -dF/dOmega under a homogeneous dilation at fixed T (Results,
// Table 1 and Fig. 3 report pressures).  p_out_h (host double[8]):
// TF, vW, NL, Hartree, loc, xc, ion, total.
template <typename T>
int Engine<T>::pressure(const void* rho, double* p_out_h, void* stream_) {
  if (!ions_set) { set_error("ofdft_structure_factor must be called before ofdft_pressure"); return OFDFT_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream_;
  int rc;
  // energies of the degree -2 / -1 terms from one evaluation
  if ((rc = eval(0, (const T*)rho, nullptr, nullptr, 0.0, 1.0, 0.0, 0.0, nullptr, st, true))) return rc;
  const double E_vW = res_h[1], E_H = res_h[3], Eion = res_h[6];
  const bool nl = use_na();
  if (nl && !p_ready && (rc = build_pressure_table(st))) return rc;
  // n~ into spec[0], (n^a)~ into spec[1], tiled layout
  Spectra<T> sp{};
  sp.s[0] = spec[0]; sp.s[1] = spec[1]; sp.nact = 2; sp.idx[0] = 0; sp.idx[1] = 1;
  ProArgs<T> pa{0, (const T*)rho, nullptr, nullptr, (T)0, (T)1, (T)cs.alpha};
  OFDFT_RUN("k_zfwd", st, (double)N * sizeof(T) + 2.0 * NH * sizeof(C), k_zfwd<T><<<grid_z, kThreads, smem_zf, st>>>(pa, sp, ph, tw_h, tw_n, n, zR, zP));
  OFDFT_RUN("k_ypass", st, 4.0 * NH * sizeof(C), k_ypass<T, -1><<<dim3(grid_y1, 2), kThreads, smem_y, st>>>(sp, pn, tw_n, n, yJ));
  OFDFT_RUN("k_xpass", st, 4.0 * NH * sizeof(C), k_xpass<T, -1><<<dim3(grid_x, 2), kThreads, smem_xp, st>>>(sp, pn, tw_n, n, xJ));
  const int gb = 4 * nsm;
  const double cy = 9.8696044010893586188344909998762 / (1.4142135623730950488016887242097 * std::pow(Te, 1.5));
  OFDFT_RUN("k_pressure_r", st, (double)N * sizeof(T), k_pressure_r<T><<<gb, 256, 0, st>>>((const T*)rho, N, (T)cy, (T)Te, cs.terms, partials, cs.fd64 ? 1 : 0, cy));
  if ((rc = sum_partials(gb, 2, 0, st))) return rc;
  const double tp = 2.0 * kPi / L;
  const C* vl = (cs.terms & OFDFT_TERM_LOC) ? vloc : nullptr;
  const double* pn_d = nl ? p_tab + (size_t)4 * (3 * h * h + 1) : nullptr;
  OFDFT_RUN("k_pressure_g", st, 3.0 * NH * sizeof(C), k_pressure_g<T><<<gb, 256, 0, st>>>(spec[0], spec[1], vl, pn_d, n, tp * tp, g2cut_loc, cs.rc * cs.rc, 1.0 / (double)N, partials));
  if ((rc = sum_partials(gb, 2, 2, st))) return rc;
  OFDFT_CK(cudaMemcpyAsync(res_h, res_d, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  OFDFT_CK(cudaStreamSynchronize(st));
  double* P = p_out_h;
  P[0] = res_h[0] / (double)N;              // (1/Omega) dV sum n T p
  P[1] = 2.0 * E_vW / (3.0 * Omega);
  P[2] = -res_h[3] / 3.0;
  P[3] = E_H / (3.0 * Omega);
  P[4] = res_h[2] / 3.0;
  P[5] = res_h[1] / (double)N;
  P[6] = Eion / (3.0 * Omega);
  P[7] = P[0] + P[1] + P[2] + P[3] + P[4] + P[5] + P[6];
  return OFDFT_OK;
}

// Ion dynamics (Methods, molecular dynamics): velocity Verlet with one
// Nose-Hoover variable in a symmetric Trotter splitting,
//   NH(dt/2)  v += dt F/(2m)  x += dt v  [electrons, F]  v += dt F/(2m)  NH(dt/2),
//   NH(h): xi += h (2K - g T)/(2Q); v *= exp(-xi h); s += xi h; xi += h (2K - g T)/(2Q),
// g = 3 N_i - 3, Q = g T tau^2; conserved H = F_min + K + Q xi^2/2 + g T s.
// Every step the electrons are minimised at the new positions starting from
// the previous density (rho_io), and the Hellmann-Feynman forces follow.
template <typename T>
int Engine<T>::md_run(void* rho_io, int start_uniform, double* pos_io, double* vel_io, const double* mass,
                      const ofdft_md_opts& o, ofdft_md_thermostat* th, int n_steps, ofdft_md_frame* frames,
                      double* q_out, double* sei_sum, double* sii_sum, void* stream_) {
  cudaStream_t st = (cudaStream_t)stream_;
  const int ni = (int)cs.Z.size();
  const bool thermo = o.T_ion > 0;
  const double g = 3.0 * ni - 3.0;
  if (thermo && (g <= 0 || !(o.tau > 0))) {
    set_error("ofdft_md_run: a thermostat needs at least 2 ions and tau > 0");
    return OFDFT_ERR_INVALID;
  }
  const double Q = thermo ? g * o.T_ion * o.tau * o.tau : 0.0;
  int rc;
  if (o.n_shells > 0 && (rc = build_shells(o.n_shells, st))) return rc;
  const size_t nc = (size_t)ni * 3;
  std::vector<double> x(pos_io, pos_io + nc), v(vel_io, vel_io + nc), F(nc), hout;
  for (auto& c : x) c -= L * std::floor(c / L);
  ofdft_result r{};
  auto electrons = [&](int uniform) -> int {
    int e;
    if ((e = set_ions(x.data(), 0, nullptr, st))) return e;
    if ((e = minimize(rho_io, uniform, o.min, &r, st))) return e;
    return forces(rho_io, F.data(), st);
  };
  auto kinetic = [&]() {
    double k = 0;
    for (size_t c = 0; c < nc; ++c) k += 0.5 * mass[c / 3] * v[c] * v[c];
    return k;
  };
  auto nh = [&](double h) {
    th->xi += 0.5 * h * (2.0 * kinetic() - g * o.T_ion) / Q;
    const double f = std::exp(-th->xi * h);
    for (auto& c : v) c *= f;
    th->s += th->xi * h;
    th->xi += 0.5 * h * (2.0 * kinetic() - g * o.T_ion) / Q;
  };
  if ((rc = electrons(start_uniform))) return rc;
  const double dt = o.dt;
  for (int step = 0; step < n_steps; ++step) {
    const std::vector<double> x0 = x, v0 = v;
    const double xi0 = th->xi, s0 = th->s;
    if (thermo) nh(0.5 * dt);
    for (size_t c = 0; c < nc; ++c) v[c] += 0.5 * dt * F[c] / mass[c / 3];
    for (size_t c = 0; c < nc; ++c) x[c] += dt * v[c];
    for (auto& c : x) c -= L * std::floor(c / L);
    if ((rc = electrons(0))) {
      // leave the state of the last completed step
      std::copy(x0.begin(), x0.end(), pos_io);
      std::copy(v0.begin(), v0.end(), vel_io);
      th->xi = xi0; th->s = s0; th->steps_done = step;
      return rc;
    }
    for (size_t c = 0; c < nc; ++c) v[c] += 0.5 * dt * F[c] / mass[c / 3];
    if (thermo) nh(0.5 * dt);
    const double K = kinetic();
    if (frames) {
      ofdft_md_frame& fr = frames[step];
      fr.e_pot = r.e.F_total;
      fr.kinetic = K;
      fr.conserved = r.e.F_total + K + (thermo ? 0.5 * Q * th->xi * th->xi + g * o.T_ion * th->s : 0.0);
      fr.xi = th->xi;
      fr.evaluations = r.evaluations;
      fr.iterations = r.iterations;
    }
    if (o.n_shells > 0) {
      if ((rc = shell_sums(rho_io, st, hout))) return rc;
      for (int k = 0; k < sh_ns; ++k) {
        sei_sum[k] += hout[3 * k] / hout[3 * k + 2];
        sii_sum[k] += hout[3 * k + 1] / ((double)ni * hout[3 * k + 2]);
      }
    }
  }
  if (o.n_shells > 0)
    for (int k = 0; k < sh_ns; ++k) q_out[k] = 2.0 * kPi / L * std::sqrt((double)sh_m2[k]);
  std::copy(x.begin(), x.end(), pos_io);
  std::copy(v.begin(), v.end(), vel_io);
  th->steps_done = n_steps;
  return OFDFT_OK;
}

}  // namespace ofdft
