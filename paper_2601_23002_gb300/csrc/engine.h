// Internal interface between the C-ABI layer (api.cu) and the per-precision
// engines (engine_f32.cu, engine_f64.cu).  Not part of the public header.
#pragma once
#include <stddef.h>
#include <cuda_runtime.h>
#include <string>
#include <vector>

#include "../../include/ofdft.h"

namespace ofdft {

struct CellSpec {
  double L;
  int n;
  std::vector<double> Z;
  double rc;
  double T;
  int terms;
  double alpha;
  bool fd64 = false;   // FP32 plans: FP64 Fermi-Dirac inversion per point
};

class IEngine {
 public:
  virtual ~IEngine() {}
  virtual int create(void* stream) = 0;
  virtual int set_ions(const double* pos, int on_device, void* S_out, void* stream) = 0;
  virtual int energy_potential(const void* rho, void* v_out, ofdft_energies* e, void* stream) = 0;
  virtual int energy_potential_async(const void* rho, void* v_out, double* e_dev, void* stream) = 0;
  virtual int minimize(void* rho_io, int start_uniform, const ofdft_min_opts& o, ofdft_result* r,
                       void* stream) = 0;
  virtual int sei_shells(const void* rho, int n_shells, double* q_out, double* s_out, void* stream) = 0;
  virtual int forces(const void* rho, double* f_out, void* stream) = 0;
  virtual int pressure(const void* rho, double* p_out, void* stream) = 0;
  virtual int md_run(void* rho_io, int start_uniform, double* pos_io, double* vel_io, const double* mass,
                     const ofdft_md_opts& o, ofdft_md_thermostat* th, int n_steps, ofdft_md_frame* frames,
                     double* q_out, double* sei_sum, double* sii_sum, void* stream) = 0;
  virtual size_t bytes() const = 0;
  virtual int autotune(void* stream, int* tile, double* us_per_eval) = 0;
  virtual int set_tiles(const int* tile) = 0;
  virtual long long grid_points() const = 0;
  // streams that calls returning before their work is done (the potential
  // without host energies, the asynchronous energies) were given; drained
  // before the plan's memory goes back to the block cache.  Every other call
  // synchronises its stream before returning.
  std::vector<void*> async_streams;
  void note_async(void* s) {
    for (void* t : async_streams) if (t == s) return;
    async_streams.push_back(s);
  }
  virtual int profile_enable(int timing) = 0;
  virtual int profile_read(ofdft_kernel_stat* out, int max, int* count) = 0;
};

// Device and pinned-host blocks for plans, kept in a process-wide cache on
// release (api.cu): cudaFree and cudaFreeHost synchronise the whole device,
// which would stall every other stream at each plan release in the serving
// loop.  A released block is reused by a later request of the same size on
// the same device; the caller releases a block only after the work that used
// it has finished.  On allocation failure the device's cached blocks are
// freed and the allocation retried.  At most kCacheCapBytes per device are
// kept; blocks beyond that are freed at once.
constexpr size_t kCacheCapBytes = (size_t)16 << 30;
cudaError_t cached_dev_alloc(void** p, size_t bytes);
void cached_dev_release(void* p, size_t bytes);
cudaError_t cached_host_alloc(void** p, size_t bytes);
void cached_host_release(void* p, size_t bytes);

IEngine* make_engine_f32(const CellSpec& c, int m_max);
IEngine* make_engine_f64(const CellSpec& c, int m_max);
size_t engine_bytes(const CellSpec& c, int precision, int m_max);

// thread-local error message shared by all layers
void set_error(const std::string& msg);

// 1-D FFT factorisation into supported radices; false if n is not supported
bool factor_radices(int n, int* radix, int* npass);
// the same number of passes, with the smallest largest radix (the z passes'
// half-length transforms: a block's 16 rows give more butterflies per stage)
bool factor_radices_balanced(int n, int* radix, int* npass);

}  // namespace ofdft
