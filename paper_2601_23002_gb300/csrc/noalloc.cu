// ofdft_sei_shells_static: the electron-ion structure factor on |q| shells
// computed without allocating any device memory.
//
// Who needs this: code that may not call cudaMalloc or any allocating routine
// while it runs -- for example a host application whose memory budget is fixed
// up front and managed by someone else, a real-time analysis hook called from
// inside another library's simulation loop, or a process where allocation is
// forbidden after start-up so that it can never fail or fragment the heap
// mid-run.  Such callers provide the density, the ion positions and the output
// arrays; every temporary lives in one fixed array of device memory that this
// file declares at file scope.
//
// The fixed array (g_sei_scratch, kScratchBytes = about 2.5 MB) is part of the
// library image: every GPU on which the library is loaded keeps it until the
// process exits, whether or not this entry point is used.  It bounds the grid
// to n <= 64 and the request to 256 shells.
//
// All calls share the one array.  Two calls whose GPU work overlaps (on
// different streams or from different threads without ordering) race on it
// and return wrong numbers; serialise them.  Nothing in it needs to start at
// zero: every call overwrites what it reads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/ofdft.h"
#include "engine.h"
#include "fft.cuh"
#include "passes.cuh"

namespace ofdft {
namespace {

constexpr int kStaticMaxN = 64;
constexpr int kStaticMaxShells = 256;
constexpr int kStaticMaxEntries = 16384;
constexpr int kMaxDevices = 64;

// byte layout of the scratch array
constexpr size_t kSpecBytes = (size_t)kStaticMaxN * kStaticMaxN * (kStaticMaxN / 2 + 1) * sizeof(double2);
constexpr size_t kOffTwN = kSpecBytes;
constexpr size_t kOffTwH = kOffTwN + kStaticMaxN * sizeof(double2);
constexpr size_t kOffIdx = kOffTwH + kStaticMaxN / 2 * sizeof(double2);
constexpr size_t kOffWgt = kOffIdx + kStaticMaxEntries * sizeof(long long);
constexpr size_t kOffPtr = kOffWgt + kStaticMaxEntries * sizeof(float);
constexpr size_t kOffM2 = kOffPtr + (kStaticMaxShells + 1) * sizeof(int);
constexpr size_t kScratchBytes = ((kOffM2 + kStaticMaxShells * sizeof(int)) + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_sei_scratch[kScratchBytes];

// Device address of g_sei_scratch in the context current on the calling
// thread.  In host code the symbol names a host-side stand-in, not device
// memory, so the address is looked up with cudaGetSymbolAddress.  The lookup
// allocates nothing and is made on every call: a module's __device__ array
// has one address per context, and a cached address would go stale when the
// caller switches contexts on the same device (driver-API code with contexts
// of its own) or resets the device.
// One call at a time per device: the calls share the device's scratch array,
// and each holds its device's lock until its stream has drained.
std::mutex g_call_mu[kMaxDevices];

int scratch_for_current_device(unsigned char** out, int* dev_out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_error(std::string("cudaGetDevice failed: ") + cudaGetErrorString(e)); return OFDFT_ERR_CUDA; }
  if (dev < 0 || dev >= kMaxDevices) { set_error("device index out of range"); return OFDFT_ERR_INVALID; }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_sei_scratch);
  if (e != cudaSuccess || !p) {
    set_error(std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    return OFDFT_ERR_CUDA;
  }
  *out = static_cast<unsigned char*>(p);
  *dev_out = dev;
  return OFDFT_OK;
}

// Waits for `st` when it goes out of scope while armed: an error return after
// work has been queued on the scratch array must not release the device's
// lock before that work has finished.
struct DrainOnExit {
  cudaStream_t st;
  bool armed = false;
  ~DrainOnExit() {
    if (armed) { cudaStreamSynchronize(st); cudaGetLastError(); }
  }
};

// Host-side staging for the tables that are copied into the scratch array
// (fixed size, per thread, so the call allocates no host memory either).
struct HostTables {
  double2 tw_n[kStaticMaxN];
  double2 tw_h[kStaticMaxN / 2];
  long long idx[kStaticMaxEntries];
  float wgt[kStaticMaxEntries];
  int ptr[kStaticMaxShells + 1];
  int m2[kStaticMaxShells];
  char present[3 * (kStaticMaxN / 2) * (kStaticMaxN / 2) + 1];
  int shell_of[3 * (kStaticMaxN / 2) * (kStaticMaxN / 2) + 1];
  int count[kStaticMaxShells];
};
thread_local HostTables t_host;

// One block per shell: S(G) = sum_I exp(-i G.R_I) evaluated at the shell's
// G vectors, and the weighted mean of Re[n_e(G) S*(G)].
__global__ void __launch_bounds__(256) k_sei_static(const double2* __restrict__ spec, const double* __restrict__ pos,
                                                    int n_ion, int n, double L, const long long* __restrict__ idx,
                                                    const float* __restrict__ wgt, const int* __restrict__ ptr,
                                                    const int* __restrict__ m2s, double scale,
                                                    double* __restrict__ q_out, double* __restrict__ s_out) {
  __shared__ double red[2 * 32];
  const int s = blockIdx.x;
  const int nh = n / 2 + 1;
  double acc[2] = {0, 0};
  for (int e = ptr[s] + threadIdx.x; e < ptr[s + 1]; e += blockDim.x) {
    const long long q = idx[e];
    const int kx = (int)(q / ((long long)n * nh));
    const int rem = (int)(q % ((long long)n * nh));
    const int ky = rem / nh, kz = rem % nh;
    const int mx = kx <= n / 2 - 1 ? kx : kx - n;
    const int my = ky <= n / 2 - 1 ? ky : ky - n;
    double sr = 0, si = 0;
    for (int I = 0; I < n_ion; ++I) {
      double fx = pos[3 * I] / L, fy = pos[3 * I + 1] / L, fz = pos[3 * I + 2] / L;
      fx -= floor(fx); fy -= floor(fy); fz -= floor(fz);
      double t = (double)mx * fx + (double)my * fy + (double)kz * fz;
      t -= rint(t);
      double sn, cs;
      sincospi(-2.0 * t, &sn, &cs);
      sr += cs; si += sn;
    }
    const double2 a = spec[q];
    const double w = (double)wgt[e];
    acc[0] += w * (a.x * sr + a.y * si) * scale;
    acc[1] += w;
  }
  double o[2];
  block_sum<2>(acc, red, o);
  if (threadIdx.x == 0) {
    q_out[s] = 2.0 * kPi / L * sqrt((double)m2s[s]);
    s_out[s] = o[0] / o[1];
  }
}

bool smooth_even(int k) {
  if (k % 2) return false;
  for (int p : {2, 3, 5})
    while (k % p == 0) k /= p;
  return k == 1;
}

}  // namespace
}  // namespace ofdft

using namespace ofdft;

extern "C" int ofdft_sei_shells_static(const double* rho, const double* pos, int n_ion, double L, int n,
                                       double n_electrons, int n_shells, double* q_out, double* s_out,
                                       void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (!rho || !pos || !q_out || !s_out) { set_error("NULL argument"); return OFDFT_ERR_INVALID; }
  if (n < 8 || n > kStaticMaxN || !smooth_even(n)) {
    set_error("ofdft_sei_shells_static: n must be even, 2,3,5-smooth and in [8, 64] (fixed scratch size)");
    return OFDFT_ERR_INVALID;
  }
  if (n_shells < 1 || n_shells > kStaticMaxShells) {
    set_error("ofdft_sei_shells_static: n_shells must be in [1, 256] (fixed scratch size)");
    return OFDFT_ERR_INVALID;
  }
  if (n_ion < 1 || !(L > 0) || !(n_electrons > 0)) { set_error("need n_ion >= 1, L > 0, n_electrons > 0"); return OFDFT_ERR_INVALID; }
  FftPlan1 pn{}, ph{};
  if (!factor_radices(n, pn.radix, &pn.npass) || !factor_radices(n / 2, ph.radix, &ph.npass)) {
    set_error("ofdft_sei_shells_static: grid size not supported by the FFT radices");
    return OFDFT_ERR_INVALID;
  }
  pn.n = n; ph.n = n / 2;
  const int h = n / 2, nh = h + 1;
  HostTables& H = t_host;
  // shells: first n_shells distinct nonzero |m|^2 on the grid
  const int m2cap = 3 * h * h;
  std::memset(H.present, 0, (size_t)(m2cap + 1));
  for (int mx = -h; mx < h; ++mx)
    for (int my = -h; my < h; ++my)
      for (int mz = 0; mz <= h; ++mz) {
        const int m2 = mx * mx + my * my + mz * mz;
        if (m2 > 0) H.present[m2] = 1;
      }
  int ns = 0;
  for (int m2 = 1; m2 <= m2cap && ns < n_shells; ++m2)
    if (H.present[m2]) { H.shell_of[m2] = ns; H.m2[ns++] = m2; }
  if (ns < n_shells) { set_error("grid has fewer distinct shells than requested"); return OFDFT_ERR_INVALID; }
  const int m2max = H.m2[ns - 1];
  for (int m2 = 0; m2 <= m2max; ++m2)
    if (!H.present[m2] || m2 == 0) H.shell_of[m2] = -1;
  // counting sort of the half-spectrum entries by shell
  std::memset(H.count, 0, sizeof(int) * (size_t)ns);
  const int r = (int)std::ceil(std::sqrt((double)m2max));
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      H.ptr[0] = 0;
      for (int i = 0; i < ns; ++i) H.ptr[i + 1] = H.ptr[i] + H.count[i];
      if (H.ptr[ns] > kStaticMaxEntries) { set_error("too many G vectors in the requested shells"); return OFDFT_ERR_INVALID; }
      std::memset(H.count, 0, sizeof(int) * (size_t)ns);
    }
    for (int mx = -std::min(r, h); mx <= std::min(r, h - 1); ++mx)
      for (int my = -std::min(r, h); my <= std::min(r, h - 1); ++my)
        for (int mz = 0; mz <= std::min(r, h); ++mz) {
          const int m2 = mx * mx + my * my + mz * mz;
          if (m2 == 0 || m2 > m2max) continue;
          const int sh = H.shell_of[m2];
          if (sh < 0) continue;
          if (pass == 1) {
            const int e = H.ptr[sh] + H.count[sh];
            const int kx = mx < 0 ? mx + n : mx, ky = my < 0 ? my + n : my;
            H.idx[e] = ((long long)kx * n + ky) * nh + mz;
            H.wgt[e] = (mz == 0 || 2 * mz == n) ? 1.0f : 2.0f;
          }
          H.count[sh]++;
        }
  }
  for (int t = 0; t < n; ++t) {
    const long double a = -2.0L * 3.14159265358979323846264338327950288L * t / n;
    H.tw_n[t] = make_double2((double)cosl(a), (double)sinl(a));
  }
  for (int t = 0; t < h; ++t) {
    const long double a = -2.0L * 3.14159265358979323846264338327950288L * t / h;
    H.tw_h[t] = make_double2((double)cosl(a), (double)sinl(a));
  }
  unsigned char* base = nullptr;
  int dev_idx = 0;
  int rc = scratch_for_current_device(&base, &dev_idx);
  if (rc) return rc;
  std::lock_guard<std::mutex> call_lock(g_call_mu[dev_idx]);   // released after the final synchronise
  DrainOnExit drain{st};                 // declared after the lock: drains before it is released
  double2* spec = reinterpret_cast<double2*>(base);
  double2* tw_n = reinterpret_cast<double2*>(base + kOffTwN);
  double2* tw_h = reinterpret_cast<double2*>(base + kOffTwH);
  long long* idx = reinterpret_cast<long long*>(base + kOffIdx);
  float* wgt = reinterpret_cast<float*>(base + kOffWgt);
  int* ptr = reinterpret_cast<int*>(base + kOffPtr);
  int* m2s = reinterpret_cast<int*>(base + kOffM2);
  const int nent = H.ptr[ns];
#define NA_CK(call)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      set_error(std::string("ofdft_sei_shells_static: ") + cudaGetErrorString(e_));          \
      return OFDFT_ERR_CUDA;                                                                 \
    }                                                                                        \
  } while (0)
  drain.armed = true;                    // from the first copy into the array on
  NA_CK(cudaMemcpyAsync(tw_n, H.tw_n, n * sizeof(double2), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(tw_h, H.tw_h, h * sizeof(double2), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(idx, H.idx, (size_t)nent * sizeof(long long), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(wgt, H.wgt, (size_t)nent * sizeof(float), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(ptr, H.ptr, (size_t)(ns + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(m2s, H.m2, (size_t)ns * sizeof(int), cudaMemcpyHostToDevice, st));
  // forward FFT of rho into the scratch spectrum (same kernels as the plans)
  const int zR = std::max(1, std::min(32, 2048 / h));
  const int zP = nh | 1;
  const int J = 8;
  // k_zfwd shared memory: two real row buffers (input and psi), then two complex FFT buffers
  const size_t smem_z = ((size_t)2 * zR * n * sizeof(double) + 15) / 16 * 16 + 2 * (size_t)zR * zP * sizeof(double2);
  const size_t smem_t = 2 * (size_t)n * J * sizeof(double2);
  // The limit belongs to the kernel function, which the plans share: raise it
  // to the device maximum instead of this call's size, so that no larger plan
  // launched later finds it lowered.
  int dev_lim = 0, dev_id = 0;
  NA_CK(cudaGetDevice(&dev_id));
  NA_CK(cudaDeviceGetAttribute(&dev_lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev_id));
  if ((size_t)dev_lim < std::max(smem_z, smem_t) + 8192) { set_error("shared memory too small"); return OFDFT_ERR_INVALID; }
  {
    const void* fs[3] = {(const void*)k_zfwd<double>, (const void*)k_ypass<double, -1>,
                         (const void*)k_xpass<double, -1>};
    for (const void* f : fs) {
      cudaFuncAttributes fa;
      NA_CK(cudaFuncGetAttributes(&fa, f));
      NA_CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dev_lim - (int)fa.sharedSizeBytes));
    }
  }
  Spectra<double> sp{};
  sp.s[0] = spec; sp.nact = 1; sp.idx[0] = 0;
  ProArgs<double> pa{0, rho, nullptr, nullptr, 0.0, 1.0, 0.5};
  const int grid_z = (n * n + zR - 1) / zR;
  k_zfwd<double><<<grid_z, 256, smem_z, st>>>(pa, sp, ph, tw_h, tw_n, n, zR, zP);
  NA_CK(cudaGetLastError());
  k_ypass<double, -1><<<dim3(n * ((nh + J - 1) / J), 1), 256, smem_t, st>>>(sp, pn, tw_n, n, J);
  NA_CK(cudaGetLastError());
  k_xpass<double, -1><<<dim3((n * nh + J - 1) / J, 1), 256, smem_t, st>>>(sp, pn, tw_n, n, J);
  NA_CK(cudaGetLastError());
  const double N = (double)n * n * n;
  const double scale = L * L * L / N / std::sqrt(n_electrons * (double)n_ion);
  k_sei_static<<<ns, 256, 0, st>>>(spec, pos, n_ion, n, L, idx, wgt, ptr, m2s, scale, q_out, s_out);
  NA_CK(cudaGetLastError());
  // the host tables above are reused by the next call on this thread
  NA_CK(cudaStreamSynchronize(st));
  drain.armed = false;
#undef NA_CK
  return OFDFT_OK;
}
