// C-ABI entry points (include/ofdft.h): argument validation, plan lifetime,
// dispatch to the FP32 or FP64 engine.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "engine.h"

namespace ofdft {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

// ---------------------------------------------------------------------------
// Block cache (see engine.h).  Device blocks are keyed by (device, size);
// pinned host blocks by size.
namespace {
struct BlockCache {
  std::mutex mu;
  std::map<std::pair<int, size_t>, std::vector<void*>> dev;
  std::map<int, size_t> dev_bytes;                 // cached bytes per device
  std::map<size_t, std::vector<void*>> host;
};
BlockCache& cache() {
  static BlockCache* c = new BlockCache();         // never destroyed: plans may outlive statics
  return *c;
}
int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}
}  // namespace

cudaError_t cached_dev_alloc(void** p, size_t bytes) {
  BlockCache& c = cache();
  const int d = current_device();
  {
    std::lock_guard<std::mutex> lock(c.mu);
    auto it = c.dev.find({d, bytes});
    if (it != c.dev.end() && !it->second.empty()) {
      *p = it->second.back();
      it->second.pop_back();
      c.dev_bytes[d] -= bytes;
      return cudaSuccess;
    }
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    // give this device's cached blocks back and try once more
    std::vector<void*> drop;
    {
      std::lock_guard<std::mutex> lock(c.mu);
      for (auto it = c.dev.begin(); it != c.dev.end(); ++it)
        if (it->first.first == d) {
          drop.insert(drop.end(), it->second.begin(), it->second.end());
          it->second.clear();
        }
      c.dev_bytes[d] = 0;
    }
    for (void* q : drop) cudaFree(q);
    e = cudaMalloc(p, bytes);
  }
  return e;
}

void cached_dev_release(void* p, size_t bytes) {
  if (!p) return;
  BlockCache& c = cache();
  const int d = current_device();
  {
    std::lock_guard<std::mutex> lock(c.mu);
    if (c.dev_bytes[d] + bytes <= kCacheCapBytes) {
      c.dev[{d, bytes}].push_back(p);
      c.dev_bytes[d] += bytes;
      return;
    }
  }
  cudaFree(p);
}

cudaError_t cached_host_alloc(void** p, size_t bytes) {
  BlockCache& c = cache();
  {
    std::lock_guard<std::mutex> lock(c.mu);
    auto it = c.host.find(bytes);
    if (it != c.host.end() && !it->second.empty()) {
      *p = it->second.back();
      it->second.pop_back();
      return cudaSuccess;
    }
  }
  return cudaMallocHost(p, bytes);
}

void cached_host_release(void* p, size_t bytes) {
  if (!p) return;
  BlockCache& c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  c.host[bytes].push_back(p);
}

// n = product of radices from {16, 12, 10, 9, 8, 6, 5, 4, 3, 2}, fewest passes.
bool factor_radices(int n, int* radix, int* npass) {
  static const int cand[] = {16, 12, 10, 9, 8, 6, 5, 4, 3, 2};
  if (n == 1) { *npass = 1; radix[0] = 1; return false; }
  for (int passes = 1; passes <= 8; ++passes) {
    // depth-first search for a factorisation with exactly `passes` factors
    int fac[8];
    bool found = false;
    auto dfs = [&](auto&& self, int rem, int depth) -> void {
      if (found) return;
      if (depth == passes) { if (rem == 1) found = true; return; }
      for (int c : cand) {
        if (rem % c == 0) {
          fac[depth] = c;
          self(self, rem / c, depth + 1);
          if (found) return;
        }
      }
    };
    dfs(dfs, n, 0);
    if (found) {
      *npass = passes;
      for (int i = 0; i < passes; ++i) radix[i] = fac[i];
      return true;
    }
  }
  return false;
}

bool factor_radices_balanced(int n, int* radix, int* npass) {
  static const int cand[] = {16, 12, 10, 9, 8, 6, 5, 4, 3, 2};
  int first[8], np = 0;
  if (!factor_radices(n, first, &np)) return false;
  // among the factorisations with the fewest passes, the smallest largest radix
  int best[8], bestmax = 1 << 30, fac[8];
  auto dfs = [&](auto&& self, int rem, int depth, int mx) -> void {
    if (depth == np) {
      if (rem == 1 && mx < bestmax) { bestmax = mx; for (int i = 0; i < np; ++i) best[i] = fac[i]; }
      return;
    }
    for (int c : cand)
      if (rem % c == 0) { fac[depth] = c; self(self, rem / c, depth + 1, mx > c ? mx : c); }
  };
  dfs(dfs, n, 0, 0);
  *npass = np;
  for (int i = 0; i < np; ++i) radix[i] = best[i];
  return true;
}

}  // namespace ofdft

using namespace ofdft;

struct ofdft_plan {
  IEngine* eng;
  int precision;
  int device;
  int n_ion;
};

static bool smooth235(int k) {
  for (int p : {2, 3, 5})
    while (k % p == 0) k /= p;
  return k == 1;
}

static int validate(const ofdft_cell* c, const ofdft_opts* o) {
  if (!c || !o) { set_error("cell and opts must not be NULL"); return OFDFT_ERR_INVALID; }
  if (!(c->L > 0) || !std::isfinite(c->L)) { set_error("L must be positive"); return OFDFT_ERR_INVALID; }
  if (c->n < 8 || c->n > 512 || !smooth235(c->n)) {
    set_error("n must be 2,3,5-smooth and in [8, 512]");
    return OFDFT_ERR_INVALID;
  }
  int rad[8], np;
  if (!factor_radices(c->n, rad, &np) || (c->n % 2 == 0 && !factor_radices(c->n / 2, rad, &np))) {
    set_error("n has no supported radix factorisation");
    return OFDFT_ERR_INVALID;
  }
  if (c->n_ion < 1 || !c->Z) { set_error("need n_ion >= 1 and Z"); return OFDFT_ERR_INVALID; }
  for (int i = 0; i < c->n_ion; ++i)
    if (!(c->Z[i] > 0) || !std::isfinite(c->Z[i])) { set_error("every Z must be positive"); return OFDFT_ERR_INVALID; }
  if (!(c->rc > 0) || !std::isfinite(c->rc)) { set_error("rc must be positive and finite"); return OFDFT_ERR_INVALID; }
  if (!(c->T > 0) || !std::isfinite(c->T)) { set_error("T must be positive"); return OFDFT_ERR_INVALID; }
  if (o->precision != OFDFT_FP64 && o->precision != OFDFT_FP32) { set_error("bad precision"); return OFDFT_ERR_INVALID; }
  if (o->terms < 0 || o->terms > OFDFT_TERMS_ALL) { set_error("bad terms mask"); return OFDFT_ERR_INVALID; }
  if (!(o->alpha > 0 && o->alpha < 1)) { set_error("alpha must be in (0, 1)"); return OFDFT_ERR_INVALID; }
  if (o->fd64 != 0 && o->fd64 != 1) { set_error("fd64 must be 0 or 1"); return OFDFT_ERR_INVALID; }
  return OFDFT_OK;
}

// Minimiser options, checked alike by the single, batched and MD entry points.
static int validate_min_opts(const ofdft_min_opts& o, const char* who) {
  if (o.m < 1 || o.m > 8 || o.max_iter < 1 || !(o.c1 > 0) || !(o.c2 > o.c1) || !(o.c2 < 1)) {
    set_error(std::string(who) + ": bad minimiser options (m in 1..8, max_iter >= 1, 0 < c1 < c2 < 1)");
    return OFDFT_ERR_INVALID;
  }
  if (!(o.tol_F_per_ion >= 0) || !(o.tol_residual >= 0)) {
    set_error(std::string(who) + ": bad minimiser options (tolerances must be >= 0, not NaN)");
    return OFDFT_ERR_INVALID;
  }
  return OFDFT_OK;
}

static CellSpec spec_of(const ofdft_cell* c, const ofdft_opts* o) {
  CellSpec s;
  s.L = c->L; s.n = c->n; s.Z.assign(c->Z, c->Z + c->n_ion); s.rc = c->rc; s.T = c->T;
  s.terms = o->terms; s.alpha = o->alpha; s.fd64 = o->fd64 != 0;
  return s;
}

extern "C" {

void ofdft_default_opts(ofdft_opts* o) {
  if (!o) return;
  o->precision = OFDFT_FP64;
  o->terms = OFDFT_TERMS_ALL;
  o->alpha = 0.5;
  o->fd64 = 0;
}

void ofdft_default_min_opts(ofdft_min_opts* o) {
  if (!o) return;
  o->tol_F_per_ion = 1e-6;
  o->tol_residual = 1e-4;
  o->m = 8;
  o->max_iter = 1000;
  o->c1 = 1e-4;
  o->c2 = 0.9;
}

const char* ofdft_last_error(void) { return g_err.c_str(); }
const char* ofdft_version(void) { return "ofdft-gb300 0.1 (sm_103a)"; }

size_t ofdft_plan_bytes(const ofdft_cell* cell, const ofdft_opts* opts) {
  if (validate(cell, opts)) return 0;
  return engine_bytes(spec_of(cell, opts), opts->precision, 8);
}

int ofdft_plan_create(const ofdft_cell* cell, const ofdft_opts* opts, void* stream, ofdft_plan** out) {
  if (!out) { set_error("out must not be NULL"); return OFDFT_ERR_INVALID; }
  *out = nullptr;
  int rc = validate(cell, opts);
  if (rc) return rc;
  ofdft_plan* p = new (std::nothrow) ofdft_plan;
  if (!p) { set_error("host allocation failed"); return OFDFT_ERR_OOM; }
  p->precision = opts->precision;
  p->n_ion = cell->n_ion;
  cudaGetDevice(&p->device);
  CellSpec s = spec_of(cell, opts);
  p->eng = opts->precision == OFDFT_FP32 ? make_engine_f32(s, 8) : make_engine_f64(s, 8);
  rc = p->eng->create(stream);
  if (rc) {
    std::string keep = ofdft_last_error();
    delete p->eng;
    delete p;
    set_error(keep);
    return rc;
  }
  *out = p;
  return OFDFT_OK;
}

void ofdft_plan_destroy(ofdft_plan* plan) {
  if (!plan) return;
  // the plan's blocks go back to its own device's cache
  int cur = 0;
  const bool have = cudaGetDevice(&cur) == cudaSuccess;
  if (have && cur != plan->device) cudaSetDevice(plan->device);
  delete plan->eng;
  if (have && cur != plan->device) cudaSetDevice(cur);
  delete plan;
}

int ofdft_structure_factor(ofdft_plan* plan, const double* pos, int pos_on_device, void* S_out, void* stream) {
  if (!plan || !pos) { set_error("plan and pos must not be NULL"); return OFDFT_ERR_INVALID; }
  return plan->eng->set_ions(pos, pos_on_device, S_out, stream);
}

int ofdft_energy_potential(ofdft_plan* plan, const void* rho, void* v_out, ofdft_energies* e_out, void* stream) {
  if (!plan || !rho) { set_error("plan and rho must not be NULL"); return OFDFT_ERR_INVALID; }
  if (!e_out) plan->eng->note_async(stream);        // returns without synchronising
  return plan->eng->energy_potential(rho, v_out, e_out, stream);
}

int ofdft_energy_potential_async(ofdft_plan* plan, const void* rho, void* v_out, double* e_dev, void* stream) {
  if (!plan || !rho || !e_dev) { set_error("plan, rho and e_dev must not be NULL"); return OFDFT_ERR_INVALID; }
  plan->eng->note_async(stream);
  return plan->eng->energy_potential_async(rho, v_out, e_dev, stream);
}

int ofdft_minimize(ofdft_plan* plan, void* rho_io, int start_uniform, const ofdft_min_opts* o, ofdft_result* r,
                   void* stream) {
  ofdft_min_opts d;
  ofdft_default_min_opts(&d);
  const ofdft_min_opts& oo = o ? *o : d;
  if (int rc = validate_min_opts(oo, "ofdft_minimize")) return rc;
  if (!plan || !rho_io) { set_error("plan and rho_io must not be NULL"); return OFDFT_ERR_INVALID; }
  return plan->eng->minimize(rho_io, start_uniform, oo, r, stream);
}

int ofdft_sei_shells(ofdft_plan* plan, const void* rho, int n_shells, double* q_out, double* s_out, void* stream) {
  if (!plan || !rho || !q_out || !s_out) { set_error("NULL argument"); return OFDFT_ERR_INVALID; }
  return plan->eng->sei_shells(rho, n_shells, q_out, s_out, stream);
}

int ofdft_forces(ofdft_plan* plan, const void* rho, double* forces_out, void* stream) {
  if (!plan || !rho || !forces_out) { set_error("NULL argument"); return OFDFT_ERR_INVALID; }
  return plan->eng->forces(rho, forces_out, stream);
}

int ofdft_pressure(ofdft_plan* plan, const void* rho, double* p_out, void* stream) {
  if (!plan || !rho || !p_out) { set_error("NULL argument"); return OFDFT_ERR_INVALID; }
  return plan->eng->pressure(rho, p_out, stream);
}

int ofdft_md_run(ofdft_plan* plan, void* rho_io, int start_uniform, double* pos_io, double* vel_io,
                 const double* mass, const ofdft_md_opts* o, ofdft_md_thermostat* th_io, int n_steps,
                 ofdft_md_frame* frames, double* q_out, double* sei_sum, double* sii_sum, void* stream) {
  if (!plan || !rho_io || !pos_io || !vel_io || !mass || !o || !th_io) { set_error("NULL argument"); return OFDFT_ERR_INVALID; }
  if (n_steps < 0 || !(o->dt > 0)) { set_error("ofdft_md_run: n_steps >= 0 and dt > 0 required"); return OFDFT_ERR_INVALID; }
  if (int rc = validate_min_opts(o->min, "ofdft_md_run")) return rc;
  if (o->n_shells > 0 && (!q_out || !sei_sum || !sii_sum)) { set_error("ofdft_md_run: shell outputs required"); return OFDFT_ERR_INVALID; }
  if (!std::isfinite(o->dt) || !std::isfinite(o->T_ion) || (o->T_ion > 0 && !(o->tau > 0 && std::isfinite(o->tau)))) {
    set_error("ofdft_md_run: dt, T_ion must be finite; a thermostat (T_ion > 0) needs a finite tau > 0");
    return OFDFT_ERR_INVALID;
  }
  {
    const int ni = plan->n_ion;
    for (int i = 0; i < ni; ++i)
      if (!(mass[i] > 0) || !std::isfinite(mass[i])) { set_error("ofdft_md_run: masses must be finite and > 0"); return OFDFT_ERR_INVALID; }
    for (int c = 0; c < 3 * ni; ++c)
      if (!std::isfinite(pos_io[c]) || !std::isfinite(vel_io[c])) {
        set_error("ofdft_md_run: positions and velocities must be finite");
        return OFDFT_ERR_INVALID;
      }
  }
  const ofdft_min_opts& m = o->min;
  if (m.m < 1 || m.m > 8 || m.max_iter < 1 || !(m.c1 > 0) || !(m.c2 > m.c1) || !(m.c2 < 1)) {
    set_error("bad minimiser options (m in 1..8, max_iter >= 1, 0 < c1 < c2 < 1)");
    return OFDFT_ERR_INVALID;
  }
  th_io->steps_done = 0;
  return plan->eng->md_run(rho_io, start_uniform, pos_io, vel_io, mass, *o, th_io, n_steps, frames, q_out,
                           sei_sum, sii_sum, stream);
}

int ofdft_profile_enable(ofdft_plan* plan, int timing) {
  if (!plan) { set_error("plan must not be NULL"); return OFDFT_ERR_INVALID; }
  return plan->eng->profile_enable(timing);
}

int ofdft_profile_read(ofdft_plan* plan, ofdft_kernel_stat* out, int max, int* count) {
  if (!plan || max < 0) { set_error("plan must not be NULL"); return OFDFT_ERR_INVALID; }
  return plan->eng->profile_read(out, max, count);
}

int ofdft_minimize_batch(ofdft_plan* const* plans, void* const* rhos, int count, int start_uniform,
                         const ofdft_min_opts* o, ofdft_result* results, int concurrency) {
  if (count < 0 || (count > 0 && (!plans || !rhos || !results)) || concurrency < 1) {
    set_error("ofdft_minimize_batch: bad arguments");
    return OFDFT_ERR_INVALID;
  }
  for (int i = 0; i < count; ++i)
    if (!plans[i] || !rhos[i]) { set_error("ofdft_minimize_batch: NULL plan or density"); return OFDFT_ERR_INVALID; }
  ofdft_min_opts d;
  ofdft_default_min_opts(&d);
  const ofdft_min_opts oo = o ? *o : d;
  if (int rc = validate_min_opts(oo, "ofdft_minimize_batch")) return rc;
  // largest grids first
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return plans[a]->eng->grid_points() > plans[b]->eng->grid_points();
  });
  std::atomic<int> next{0};
  std::vector<int> rcs(count, OFDFT_OK);
  std::vector<std::string> errs(count);
  const int nw = std::min(concurrency, std::max(count, 1));
  auto worker = [&]() {
    cudaStream_t st = nullptr;
    int dev_cur = -1;
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= count) break;
      const int i = order[k];
      if (plans[i]->device != dev_cur) {
        if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); st = nullptr; }
        cudaSetDevice(plans[i]->device);
        dev_cur = plans[i]->device;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
          rcs[i] = OFDFT_ERR_CUDA;
          errs[i] = "stream creation failed";
          st = nullptr;
          continue;
        }
      }
      rcs[i] = plans[i]->eng->minimize(rhos[i], start_uniform, oo, &results[i], st);
      if (rcs[i]) errs[i] = ofdft_last_error();
    }
    if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
  };
  std::vector<std::thread> pool;
  for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  int ret = OFDFT_OK;
  for (int i = 0; i < count; ++i) {
    if (rcs[i] && rcs[i] != OFDFT_ERR_NOT_CONVERGED) { set_error(errs[i]); return rcs[i]; }
    if (rcs[i] == OFDFT_ERR_NOT_CONVERGED) { ret = OFDFT_ERR_NOT_CONVERGED; set_error(errs[i]); }
  }
  return ret;
}

static std::mutex g_tile_mu;
static std::map<std::tuple<int, int>, std::vector<int>> g_tiles;   // (n, precision) -> tiles

int ofdft_autotune(ofdft_plan* plan, void* stream, int* tile, double* us_per_eval) {
  if (!plan) { set_error("plan must not be NULL"); return OFDFT_ERR_INVALID; }
  const auto key = std::make_tuple((int)std::lround(std::cbrt((double)plan->eng->grid_points())), plan->precision);
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tiles.find(key);
    if (it != g_tiles.end()) {
      int rc = plan->eng->set_tiles(it->second.data());
      if (rc == OFDFT_OK) {
        if (tile) std::copy(it->second.begin(), it->second.end(), tile);
        if (us_per_eval) *us_per_eval = -1.0;   // reused, not timed
      }
      return rc;
    }
  }
  int t[3] = {0, 0, 0};
  int rc = plan->eng->autotune(stream, t, us_per_eval);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    g_tiles[key] = std::vector<int>(t, t + 3);
  }
  if (tile) std::copy(t, t + 3, tile);
  return OFDFT_OK;
}

int ofdft_set_tiles(ofdft_plan* plan, const int* tile) {
  if (!plan || !tile) { set_error("plan and tile must not be NULL"); return OFDFT_ERR_INVALID; }
  return plan->eng->set_tiles(tile);
}

}  // extern "C"
