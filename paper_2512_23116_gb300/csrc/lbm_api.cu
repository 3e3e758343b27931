// C ABI of the GB300 lattice Boltzmann library (declared in include/lbm.h).
//
// Host side only: parameter derivation (Sec. 3.1, Eqs. bare_viscosity and
// forcing_amplitude), device memory, tile decomposition, the step schedule
// (AA parity, fused statistics every stats_every steps) replayed from CUDA
// graphs, the autotuner, and the host-side finishing of the FP64 reductions
// (means, percentiles, derived scales of Eqs. integral_length_scale -
// dissipation_rate).  Every per-cell operation runs in the kernels.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_check.cuh"
#include "lbm_internal.h"
#include "lbm_kernels.h"

#define LBM_API extern "C" __attribute__((visibility("default")))

namespace {

using namespace lbm;

constexpr int kRingCap = 1024;
constexpr int kMinHistWindow = 256;  // fewer histogram bins than this in shared memory: all global
constexpr int64_t kChunkCells = 4 << 20;
constexpr double kPi = 3.14159265358979323846;

thread_local std::string g_create_error;

struct Inst {
  lbm_params p;
  double nu0 = 0, s_nu0 = 0, F0 = 0, C = 0;
  int nxp = 0;
  int64_t ncell = 0;
  void* f = nullptr;
  size_t f_bytes = 0;
  float* tables = nullptr;  // fx_of_y[ny], fy_of_z[nz], fz_of_x[nx]
  int hist_bins = 4096;
  double hist_max = 0.02;
  int rows = 1;
  int64_t tile_begin = 0, tile_end = 0;
  // lazily allocated diagnostic buffers
  float* u = nullptr;       // [3][ncell]
  float* aux = nullptr;     // [3][ncell]
  float* plane = nullptr;   // largest plane
  uint32_t* hist = nullptr; // [hist_bins + 1]
  bool has_plan = false;
  cufftHandle plan = 0;
  void* fft_out = nullptr;
  uint64_t rec_read = 0;
  // what the diagnostic buffers hold: u of state version u_version; the
  // spectrum (shells 0..spec_kmax) of state version spec_version
  uint64_t u_version = 0, spec_version = 0;
  int spec_kmax = -1;
  std::vector<double> spec_E;
};

struct GraphKey {
  int64_t phase, len;
  bool operator<(const GraphKey& o) const { return phase != o.phase ? phase < o.phase : len < o.len; }
};

}  // namespace

struct lbm_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int precision = 0;
  size_t esize = 4;
  int num_sms = 0;
  int stats_every = 0;
  std::vector<Inst> inst;
  InstDesc* d_desc = nullptr;
  std::vector<InstDesc> h_desc;
  int64_t total_tiles = 0;
  int64_t t = 0;
  uint64_t version = 1;  // bumped by every call that changes the populations
  // kernel configuration
  int kind = 1, rows_fixed = 0, stages = 0, threads = 256, bps = 1, grid = 1, smem = 0;
  int slot_bytes = 0;  // TMA shared-memory slot layout (kSlot3, kSlot2) or 0
  int layout = 0;      // population array: 0 population-major, 1 row-interleaved
  int tile_bytes_max = 0;
  // reductions
  double* d_partials = nullptr;
  size_t partials_elems = 0;
  double* d_results = nullptr;
  double* d_ring = nullptr;
  unsigned long long* d_seq = nullptr;
  std::vector<int64_t> rec_steps;  // time of record k (k = device sequence number)
  uint32_t* d_err = nullptr;
  void* d_scratch = nullptr;
  size_t scratch_bytes = 0;
  double* d_spec = nullptr;
  size_t spec_elems = 0;
  std::map<GraphKey, cudaGraphExec_t> graphs;
  bool use_graphs = true;
  long long wait_ns = 2000000000ll;  // bound of device-side waits
  int inject_withhold = 0;           // test hook, consumed by the next TMA step launch
  long long inject_wait_ns = 0;
  std::string err;
};

namespace {

int fail(lbm_t h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_create_error = buf;
  return code;
}

#define CK(h, call)                                                                   \
  do {                                                                                \
    cudaError_t e__ = (call);                                                         \
    if (e__ != cudaSuccess)                                                           \
      return fail((h), e__ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, \
                  "%s: %s", #call, cudaGetErrorString(e__));                          \
  } while (0)

#define CKF(h, call)                                                         \
  do {                                                                       \
    cufftResult r__ = (call);                                                \
    if (r__ != CUFFT_SUCCESS)                                                \
      return fail((h), LBM_ERR_CUDA, "%s: cuFFT error %d", #call, (int)r__); \
  } while (0)

int elems_per_16b(int precision) { return precision == LBM_FP32 ? 4 : 8; }

int validate(const lbm_params& p, std::string& why) {
  char b[256];
  if (p.nx < 1 || p.ny < 1 || p.nz < 1) {
    snprintf(b, sizeof b, "lattice size %dx%dx%d: each must be >= 1", p.nx, p.ny, p.nz);
    why = b;
    return LBM_ERR_INVALID_ARG;
  }
  if ((int64_t)p.nx * p.ny * p.nz > (int64_t)1 << 33) {
    why = "lattice larger than 2^33 cells";
    return LBM_ERR_INVALID_ARG;
  }
  if (p.nx > 8192) {
    why = "nx > 8192 is not supported";
    return LBM_ERR_UNSUPPORTED;
  }
  if (p.precision < 0 || p.precision > 2) { why = "unknown precision"; return LBM_ERR_INVALID_ARG; }
  if (p.force_mode < 0 || p.force_mode > 3) { why = "unknown force_mode"; return LBM_ERR_INVALID_ARG; }
  if (!(p.cs >= 0.0) || !std::isfinite(p.cs)) { why = "Smagorinsky constant must be finite and >= 0"; return LBM_ERR_INVALID_ARG; }
  if (!(p.nu0 > 0.0) && !(p.re > 0.0 && p.u0 > 0.0)) {
    why = "nu0 <= 0 needs re > 0 and u0 > 0 to derive it";
    return LBM_ERR_INVALID_ARG;
  }
  if (p.stats_every < 0) { why = "stats_every < 0"; return LBM_ERR_INVALID_ARG; }
  if (p.hist_bins < 0 || p.hist_bins > (1 << 16)) { why = "hist_bins out of [0, 65536]"; return LBM_ERR_INVALID_ARG; }
  if (p.kernel < 0 || p.kernel > 2) { why = "unknown kernel kind"; return LBM_ERR_INVALID_ARG; }
  if (p.tile_rows < 0) { why = "tile_rows < 0"; return LBM_ERR_INVALID_ARG; }
  if (p.strain_mode < 0 || p.strain_mode > 1) { why = "strain_mode must be 0 or 1"; return LBM_ERR_INVALID_ARG; }
  if (p.layout < 0 || p.layout > 2) { why = "layout must be 0, 1 or 2"; return LBM_ERR_INVALID_ARG; }
  if (p.tma_slots < 0 || p.tma_slots > 2) { why = "tma_slots must be 0, 1 or 2"; return LBM_ERR_INVALID_ARG; }
  if (p.row_align != 0 && (p.row_align < 16 || p.row_align > 65536 || (p.row_align & (p.row_align - 1)))) {
    why = "row_align must be 0 or a power of two in [16, 65536]";
    return LBM_ERR_INVALID_ARG;
  }
  if (p.stages < 0 || p.stages > 6) { why = "stages out of [0, 6]"; return LBM_ERR_INVALID_ARG; }
  if (p.threads != 0 && (p.threads < 64 || p.threads > 512 || (p.threads & 31))) {
    why = "threads must be 0 or a multiple of 32 in [64, 512]";
    return LBM_ERR_INVALID_ARG;
  }
  if (!std::isfinite(p.body_force[0]) || !std::isfinite(p.body_force[1]) || !std::isfinite(p.body_force[2])) {
    why = "non-finite body force";
    return LBM_ERR_INVALID_ARG;
  }
  return LBM_OK;
}

void derive(Inst& I) {
  const lbm_params& p = I.p;
  // Sec. 3.1: Re = U0 Nx / nu0.
  I.nu0 = p.nu0 > 0.0 ? p.nu0 : p.u0 * p.nx / p.re;
  // Eq. (bare_viscosity): nu0 = cs^2 (1/s_nu - 1/2), cs^2 = 1/3.
  I.s_nu0 = 1.0 / (0.5 + 3.0 * I.nu0);
  // Eq. (forcing_amplitude): F0 = Cf rho U0^2 / Nx with rho = rho0 = 1.
  I.F0 = p.f0 > 0.0 ? p.f0 : p.cf * p.u0 * p.u0 / p.nx;
  I.C = p.cs;
  I.hist_bins = p.hist_bins > 0 ? p.hist_bins : 4096;
  I.hist_max = p.hist_max > 0.0 ? p.hist_max : 0.02;
  const int esz = p.precision == LBM_FP32 ? 4 : 2;
  const int align_elems = std::max(elems_per_16b(p.precision), (p.row_align > 0 ? p.row_align : 16) / esz);
  I.nxp = (p.nx + align_elems - 1) / align_elems * align_elems;
  I.ncell = (int64_t)p.nx * p.ny * p.nz;
}

std::vector<float> force_tables(const Inst& I) {
  const lbm_params& p = I.p;
  std::vector<float> t((size_t)p.ny + p.nz + p.nx, 0.0f);
  const bool sin_x = p.force_mode == LBM_FORCE_PAPER_SIN || p.force_mode == LBM_FORCE_KOLMOGOROV;
  const bool sin_yz = p.force_mode == LBM_FORCE_PAPER_SIN;
  // Eq. (forcing_pattern): Fx(j) = F0 sin(2 pi j / Ny), Fy(k) = F0 sin(2 pi k / Nz),
  // Fz(i) = F0 sin(2 pi i / Nx), with (i, j, k) = (x, y, z).
  for (int y = 0; y < p.ny; ++y) t[y] = sin_x ? (float)(I.F0 * std::sin(2.0 * kPi * y / p.ny)) : 0.f;
  for (int z = 0; z < p.nz; ++z) t[p.ny + z] = sin_yz ? (float)(I.F0 * std::sin(2.0 * kPi * z / p.nz)) : 0.f;
  for (int x = 0; x < p.nx; ++x) t[p.ny + p.nz + x] = sin_yz ? (float)(I.F0 * std::sin(2.0 * kPi * x / p.nx)) : 0.f;
  return t;
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

int ensure_scratch(lbm_t h, size_t bytes) {
  if (h->scratch_bytes >= bytes) return LBM_OK;
  if (h->d_scratch) cudaFree(h->d_scratch);
  h->d_scratch = nullptr;
  h->scratch_bytes = 0;
  CK(h, cudaMalloc(&h->d_scratch, bytes));
  h->scratch_bytes = bytes;
  return LBM_OK;
}

void clear_graphs(lbm_t h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
}

// Blocks of the read-only statistics pass: the direct kernel (256 threads) at
// full occupancy.
int diag_grid(lbm_t h) {
  return h->num_sms * std::max(1, direct_max_blocks_per_sm(h->precision, 256));
}

// Tile decomposition for the current configuration; uploads the descriptor table.
int build_tiles(lbm_t h) {
  int64_t tile = 0;
  h->h_desc.resize(h->inst.size());
  for (size_t i = 0; i < h->inst.size(); ++i) {
    Inst& I = h->inst[i];
    const lbm_params& p = I.p;
    int R;
    const int64_t row_bytes = (int64_t)19 * I.nxp * (int64_t)h->esize;
    if (h->kind == 2) {
      // a TMA stage holds at most tile_bytes_max bytes (19 segments of R x nxp values)
      const int64_t cap = h->tile_bytes_max / row_bytes;
      if (cap < 1) return fail(h, LBM_ERR_UNSUPPORTED, "an x-line of instance %zu does not fit a stage", i);
      R = (int)(h->rows_fixed > 0 ? std::min<int64_t>(h->rows_fixed, cap) : cap);
    } else {
      R = h->rows_fixed > 0 ? h->rows_fixed : std::max(1, (1024 + p.nx - 1) / p.nx);
    }
    R = std::max(1, std::min(R, p.ny));
    I.rows = R;
    const int tpp = (p.ny + R - 1) / R;
    I.tile_begin = tile;
    tile += (int64_t)tpp * p.nz;
    I.tile_end = tile;
    InstDesc& d = h->h_desc[i];
    d.f = I.f;
    d.fx_of_y = I.tables;
    d.fy_of_z = I.tables + p.ny;
    d.fz_of_x = I.tables + p.ny + p.nz;
    d.fconst[0] = p.force_mode == LBM_FORCE_CONST ? (float)p.body_force[0] : 0.f;
    d.fconst[1] = p.force_mode == LBM_FORCE_CONST ? (float)p.body_force[1] : 0.f;
    d.fconst[2] = p.force_mode == LBM_FORCE_CONST ? (float)p.body_force[2] : 0.f;
    d.nu0 = (float)I.nu0;
    d.s_nu0 = (float)I.s_nu0;
    d.C = (float)I.C;
    d.strain_mode = p.strain_mode;
    d.nx = p.nx;
    d.ny = p.ny;
    d.nz = p.nz;
    d.nxp = I.nxp;
    {
      const int e16 = elems_per_16b(h->precision);
      d.row_copy_bytes = (p.nx + e16 - 1) / e16 * e16 * (int)h->esize;
    }
    if (h->layout == 0) {  // [19][nz][ny][nxp]
      d.slot_stride = (int64_t)p.nz * p.ny * I.nxp;
      d.row_stride = I.nxp;
      d.slot_grouped = 0;
    } else {  // [nz][ny][19][nxp], slots of a cell row in grouped order
      d.slot_stride = I.nxp;
      d.row_stride = (int64_t)19 * I.nxp;
      d.slot_grouped = 1;
    }
    d.plane_stride = d.row_stride * p.ny;
    d.rows = R;
    d.tiles_per_plane = tpp;
    d.tile_begin = I.tile_begin;
    d.tile_end = I.tile_end;
    d.f_elems = (int64_t)(I.f_bytes / h->esize);
  }
  h->total_tiles = tile;
  CK(h, cudaMemcpyAsync(h->d_desc, h->h_desc.data(), sizeof(InstDesc) * h->h_desc.size(),
                        cudaMemcpyHostToDevice, h->stream));
  // partials for every block and instance
  // block partials of a step with statistics (h->grid blocks) or of the
  // statistics pass (diag_grid blocks)
  const size_t need = (size_t)h->inst.size() * (size_t)std::max(h->grid, diag_grid(h)) * kNP;
  if (need > h->partials_elems) {
    if (h->d_partials) cudaFree(h->d_partials);
    h->d_partials = nullptr;
    CK(h, cudaMalloc(&h->d_partials, need * sizeof(double)));
    h->partials_elems = need;
  }
  clear_graphs(h);
  return LBM_OK;
}

LaunchArgs base_args(lbm_t h) {
  LaunchArgs la{};
  la.insts = h->d_desc;
  la.ninst = (int)h->inst.size();
  la.tile_lo = 0;
  la.tile_hi = h->total_tiles;
  la.precision = h->precision;
  la.sa.partials = h->d_partials;
  la.sa.grid = h->grid;
  la.grid = h->grid;
  la.threads = h->threads;
  la.stages = h->stages;
  la.slot_bytes = (h->kind == 2 && h->slot_bytes == 0 && h->layout == 1) ? kSlotGrouped : h->slot_bytes;
  la.smem_bytes = h->smem;
  la.tile_bytes_max = h->tile_bytes_max;
  la.err = h->d_err;
  la.wait_ns = h->wait_ns;
  la.withhold_first_load = 0;
  return la;
}

cudaError_t launch_step(lbm_t h, const LaunchArgs& la) {
  if (h->kind != 2) return launch_step_direct(la, h->stream);
  if (h->inject_withhold) {
    LaunchArgs li = la;
    li.withhold_first_load = 1;
    li.wait_ns = h->inject_wait_ns;
    h->inject_withhold = 0;
    return launch_step_tma(li, h->stream);
  }
  return launch_step_tma(la, h->stream);
}

// Enqueue steps t0 .. t0 + n - 1 (no host state change).
int enqueue_steps(lbm_t h, int64_t t0, int64_t n) {
  for (int64_t k = 0; k < n; ++k) {
    const int64_t t = t0 + k;
    const bool stats = h->stats_every > 0 && (t % h->stats_every) == 0;
    LaunchArgs la = base_args(h);
    la.odd = (t & 1) != 0;
    la.mode = stats ? MODE_STEP_STATS : MODE_STEP;
    if (stats)
      CK(h, cudaMemsetAsync(h->d_partials, 0, h->partials_elems * sizeof(double), h->stream));
    CK(h, launch_step(h, la));
    if (stats)
      CK(h, launch_finish(h->d_partials, (int)h->inst.size(), h->grid, h->d_results, h->d_ring,
                          h->d_seq, kRingCap, h->d_err, h->stream));
  }
  return LBM_OK;
}

int64_t schedule_period(lbm_t h) {
  if (h->stats_every <= 0) return 2;
  int64_t a = 2, b = h->stats_every;
  while (b) {
    int64_t r = a % b;
    a = b;
    b = r;
  }
  return 2 / a * h->stats_every;  // lcm(2, stats_every)
}

int run_steps(lbm_t h, int64_t n) {
  if (n > 0) ++h->version;
  int64_t done = 0;
  const int64_t chunk = 32;
  while (done < n) {
    const int64_t len = std::min(chunk, n - done);
    const int64_t t0 = h->t;
    int rc;
    if (h->use_graphs && len == chunk) {
      GraphKey key{t0 % schedule_period(h), len};
      auto it = h->graphs.find(key);
      if (it == h->graphs.end()) {
        cudaGraph_t g = nullptr;
        const bool pending = cudaPeekAtLastError() != cudaSuccess;  // the caller's, left alone
        CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_steps(h, t0, len);
        cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
        if (rc != LBM_OK) {
          if (g) cudaGraphDestroy(g);
          // the invalidated capture's own error; the cause is in h->err
          if (!pending) (void)cudaGetLastError();
          return rc;
        }
        CK(h, ce);
        cudaGraphExec_t ex = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        CK(h, ie);
        it = h->graphs.emplace(key, ex).first;
      }
      CK(h, cudaGraphLaunch(it->second, h->stream));
    } else {
      rc = enqueue_steps(h, t0, len);
      if (rc != LBM_OK) return rc;
    }
    for (int64_t k = 0; k < len; ++k) {
      const int64_t t = t0 + k;
      if (h->stats_every > 0 && t % h->stats_every == 0) h->rec_steps.push_back(t);
    }
    h->t += len;
    done += len;
  }
  return LBM_OK;
}

int check_err(lbm_t h) {
  uint32_t e = 0;
  CK(h, cudaMemcpyAsync(&e, h->d_err, sizeof e, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  if (kBoundsCheck) {
    const uint32_t b = bounds_word_tma() | bounds_word_direct() | bounds_word_aux() | bounds_word_random();
    if (b) return fail(h, LBM_ERR_CUDA, "device bounds check failed (checked build; word %u)", b);
  }
  if (e) {
    CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (e & ERR_DRAIN)
      return fail(h, LBM_ERR_TIMEOUT,
                  "a device-side wait of the step kernel gave up and its copies in flight did not land "
                  "within the drain bound (error word %u)", e);
    if (e & ERR_TIMEOUT)
      return fail(h, LBM_ERR_TIMEOUT, "a device-side wait of the step kernel gave up (error word %u)", e);
    return fail(h, LBM_ERR_UNSTABLE, "non-finite values in the statistics (error word %u)", e);
  }
  return LBM_OK;
}

// Read-only pass of the step kernel over instance i: fills the requested
// per-cell outputs and the block partials, then reduces them into d_results.
int diag_pass(lbm_t h, int i, bool want_u, bool want_aux, int plane_axis, int plane_index,
              bool want_hist) {
  Inst& I = h->inst[i];
  if (want_u && !I.u) CK(h, cudaMalloc(&I.u, sizeof(float) * 3 * (size_t)I.ncell));
  if (want_aux && !I.aux) CK(h, cudaMalloc(&I.aux, sizeof(float) * 3 * (size_t)I.ncell));
  if (plane_axis >= 0 && !I.plane) {
    const lbm_params& p = I.p;
    size_t m = std::max({(size_t)p.ny * p.nz, (size_t)p.nx * p.nz, (size_t)p.nx * p.ny});
    CK(h, cudaMalloc(&I.plane, sizeof(float) * m));
  }
  if (want_hist && !I.hist) CK(h, cudaMalloc(&I.hist, sizeof(uint32_t) * (I.hist_bins + 1)));
  if (want_hist) CK(h, cudaMemsetAsync(I.hist, 0, sizeof(uint32_t) * (I.hist_bins + 1), h->stream));
  LaunchArgs la = base_args(h);
  la.tile_lo = I.tile_begin;
  la.tile_hi = I.tile_end;
  // a z-plane alone (no other output): only that plane's tiles (tiles run
  // plane by plane), and no reduction of the block partials, which then
  // cover the plane only
  const bool plane_only = plane_axis == 2 && !want_u && !want_aux && !want_hist;
  if (plane_only) {
    const int64_t tpp = (I.p.ny + I.rows - 1) / I.rows;
    la.tile_lo = I.tile_begin + (int64_t)plane_index * tpp;
    la.tile_hi = la.tile_lo + tpp;
  }
  la.odd = (h->t & 1) != 0;
  la.mode = MODE_DIAG;
  la.dout.u = want_u ? I.u : nullptr;
  la.dout.aux = want_aux ? I.aux : nullptr;
  la.dout.plane = plane_axis >= 0 ? I.plane : nullptr;
  la.dout.plane_axis = plane_axis;
  la.dout.plane_index = plane_index;
  la.dout.hist = want_hist ? I.hist : nullptr;
  la.dout.hist_bins = I.hist_bins;
  la.dout.hist_scale = (float)(I.hist_bins / I.hist_max);
  CK(h, cudaMemsetAsync(h->d_partials, 0, h->partials_elems * sizeof(double), h->stream));
  // The TMA kernel's read-only variant when the handle runs the TMA kernel
  // (its copy pipeline keeps the loads in flight during the collision
  // arithmetic; the theta histogram goes behind the Fz table in shared memory
  // when it fits), else the direct kernel at full occupancy.
  int grid = 0;
  if (h->kind == 2) {
    LaunchArgs lt = la;
    // as many histogram bins as fit behind the stages, from the bin of theta
    // = 3 nu0 up (theta = 3 nu0 + 3 C |S| is never below it; one bin of
    // margin for rounding, and a cell outside the window is still counted,
    // in global memory)
    const double b3 = 3.0 * I.nu0 * I.hist_bins / I.hist_max;  // bin of theta = 3 nu0
    const int lo = b3 >= (double)I.hist_bins ? I.hist_bins : std::max(0, (int)b3 - 1);
    const int win = std::min(I.hist_bins + 1 - lo, (tma_diag_smem_limit(h->precision) - h->smem) / 4);
    const int smem_hist = (h->smem + 4 * win + 15) / 16 * 16;
    if (want_hist && win >= kMinHistWindow && tma_prepare(h->precision, smem_hist) == cudaSuccess) {
      lt.hist_smem = h->smem;
      lt.hist_lo = lo;
      lt.hist_win = win;
      lt.smem_bytes = smem_hist;
    }
    // the pass is bound by its consumers' arithmetic, not by the copies: as
    // many consumer warps as fit (the tiles do not depend on the thread count)
    for (int th : {512, 384, h->threads}) {
      if (tma_max_blocks_per_sm(h->precision, lt.slot_bytes, th, lt.smem_bytes, true) >= 1) {
        lt.threads = th;
        break;
      }
    }
    const int bps = tma_max_blocks_per_sm(h->precision, lt.slot_bytes, lt.threads, lt.smem_bytes, true);
    const int cap = (int)(h->partials_elems / ((size_t)h->inst.size() * kNP));
    grid = std::min(h->num_sms * bps, cap);
    if (grid > 0) {
      lt.grid = grid;
      lt.sa.grid = grid;
      CK(h, launch_step_tma(lt, h->stream));
    }
  }
  if (grid == 0) {
    LaunchArgs ld = la;
    ld.threads = 256;
    ld.grid = grid = diag_grid(h);
    ld.sa.grid = ld.grid;
    CK(h, launch_step_direct(ld, h->stream));
  }
  if (!plane_only)
    CK(h, launch_finish(h->d_partials, (int)h->inst.size(), grid, h->d_results, nullptr, nullptr, 0, h->d_err,
                        h->stream));
  if (want_u) I.u_version = h->version;
  return LBM_OK;
}

void fill_from_sums(lbm_stats_t* out, const double* r, const Inst& I, int64_t t) {
  const double n = r[P_CELLS];
  out->step = t;
  out->cells = (int64_t)n;
  out->mass = r[P_DRHO];
  out->momentum[0] = r[P_MX];
  out->momentum[1] = r[P_MY];
  out->momentum[2] = r[P_MZ];
  out->E_k = 0.5 * r[P_UU] / n;
  out->inj = r[P_FU] / n;
  out->eps0 = I.nu0 * r[P_SS] / n;      // 2 nu0 <S_ij S_ij>, S_ij S_ij = |S|^2 / 2
  out->eps_sgs = r[P_NUTSS] / n;        // 2 <nu_t S_ij S_ij>
  for (int k = 0; k < 6; ++k) out->uu[k] = r[P_XX + k] / n;
  out->theta_mean = r[P_TH] / n;
  out->theta_var = std::max(0.0, r[P_TH2] / n - out->theta_mean * out->theta_mean);
  out->theta_min = r[P_THMIN];
  out->theta_max = r[P_THMAX];
  // Eq. (Kt_definition): K_t = (tau_e - 1/2) sqrt(3) dx / l with l = dx.
  out->Kt_mean = std::sqrt(3.0) * out->theta_mean;
  out->Kt_var = 3.0 * out->theta_var;
  // isotropy of the Reynolds stresses (Sec. 3.2): b_ij, its invariants, Lumley (xi, eta)
  const double tr = out->uu[0] + out->uu[1] + out->uu[2];
  if (tr > 0.0) {
    double B[3][3];
    const int ij[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int k = 0; k < 6; ++k) {
      const int i = ij[k][0], j = ij[k][1];
      B[i][j] = B[j][i] = out->uu[k] / tr - (i == j ? 1.0 / 3.0 : 0.0);
      out->b[k] = B[i][j];
    }
    for (int i = 0; i < 3; ++i) out->E_frac[i] = out->uu[i] / tr;
    double bb = 0.0, bbb = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        bb += B[i][j] * B[j][i];
        for (int k = 0; k < 3; ++k) bbb += B[i][j] * B[j][k] * B[k][i];
      }
    out->II_b = -0.5 * bb;
    out->III_b = bbb / 3.0;
    out->lumley_xi = std::cbrt(out->III_b / 2.0);
    out->lumley_eta = std::sqrt(std::max(0.0, -out->II_b / 3.0));
  }
}

// Exact integer shell s with s - 1/2 <= sqrt(K) < s + 1/2.
int max_shell(int nx, int ny, int nz) {
  const long long K = (long long)(nx / 2) * (nx / 2) + (long long)(ny / 2) * (ny / 2) +
                      (long long)(nz / 2) * (nz / 2);
  long long r = (long long)std::sqrt((double)K);
  while (r * r > K) --r;
  while ((r + 1) * (r + 1) <= K) ++r;
  return (int)(K > r * r + r ? r + 1 : r);
}

int spectrum_device(lbm_t h, int i, int kmax, double* host_E) {
  Inst& I = h->inst[i];
  const lbm_params& p = I.p;
  if (I.spec_version == h->version && I.spec_kmax >= kmax) {  // this state's spectrum is at hand
    std::copy(I.spec_E.begin(), I.spec_E.begin() + kmax + 1, host_E);
    return LBM_OK;
  }
  if (!I.has_plan) {
    CKF(h, cufftPlan3d(&I.plan, p.nz, p.ny, p.nx, CUFFT_R2C));
    I.has_plan = true;
    CK(h, cudaMalloc(&I.fft_out, sizeof(float) * 2 * (size_t)p.nz * p.ny * (p.nx / 2 + 1)));
  }
  CKF(h, cufftSetStream(I.plan, h->stream));
  const int blocks = std::min(2 * h->num_sms, 1024);
  const size_t need = (size_t)blocks * (kmax + 1) + (kmax + 1);
  if (need > h->spec_elems) {
    if (h->d_spec) cudaFree(h->d_spec);
    h->d_spec = nullptr;
    CK(h, cudaMalloc(&h->d_spec, need * sizeof(double)));
    h->spec_elems = need;
  }
  CK(h, cudaMemsetAsync(h->d_spec, 0, need * sizeof(double), h->stream));
  for (int d = 0; d < 3; ++d) {
    CKF(h, cufftExecR2C(I.plan, I.u + (size_t)d * I.ncell, static_cast<cufftComplex*>(I.fft_out)));
    CK(h, launch_spec_bin(I.fft_out, p.nx, p.ny, p.nz, kmax, h->d_spec, blocks, h->stream));
  }
  double* Edev = h->d_spec + (size_t)blocks * (kmax + 1);
  CK(h, launch_spec_finish(h->d_spec, blocks, kmax, Edev, h->stream));
  CK(h, cudaMemcpyAsync(host_E, Edev, sizeof(double) * (kmax + 1), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  I.spec_E.assign(host_E, host_E + kmax + 1);
  I.spec_kmax = kmax;
  I.spec_version = h->version;
  return LBM_OK;
}

std::vector<int> separations(int n) {
  std::vector<int> r;
  for (int k = 1; k <= n / 2; k *= 2) {
    r.push_back(k);
    if (k >= 2 && 3 * k / 2 <= n / 2) r.push_back(3 * k / 2);
  }
  std::sort(r.begin(), r.end());
  r.erase(std::unique(r.begin(), r.end()), r.end());
  return r;
}

int choose_config(lbm_t h, const lbm_params& p0);

int alloc_common(lbm_t h) {
  CK(h, cudaMalloc(&h->d_desc, sizeof(InstDesc) * h->inst.size()));
  CK(h, cudaMalloc(&h->d_results, sizeof(double) * kNP * h->inst.size()));
  CK(h, cudaMalloc(&h->d_ring, sizeof(double) * kNP * h->inst.size() * kRingCap));
  CK(h, cudaMalloc(&h->d_seq, 2 * sizeof(unsigned long long)));
  CK(h, cudaMalloc(&h->d_err, sizeof(uint32_t)));
  CK(h, cudaMemsetAsync(h->d_seq, 0, 2 * sizeof(unsigned long long), h->stream));
  CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), h->stream));
  return LBM_OK;
}

void release(lbm_t h) {
  if (!h) return;
  clear_graphs(h);
  for (Inst& I : h->inst) {
    cudaFree(I.f);
    cudaFree(I.tables);
    cudaFree(I.u);
    cudaFree(I.aux);
    cudaFree(I.plane);
    cudaFree(I.hist);
    cudaFree(I.fft_out);
    if (I.has_plan) cufftDestroy(I.plan);
  }
  cudaFree(h->d_desc);
  cudaFree(h->d_partials);
  cudaFree(h->d_results);
  cudaFree(h->d_ring);
  cudaFree(h->d_seq);
  cudaFree(h->d_err);
  cudaFree(h->d_scratch);
  cudaFree(h->d_spec);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int create_impl(const lbm_params* params, int count, lbm_t* out) {
  if (!params || !out || count < 1) return fail(nullptr, LBM_ERR_INVALID_ARG, "null argument or count < 1");
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    std::string why;
    int rc = validate(params[i], why);
    if (rc != LBM_OK) return fail(nullptr, rc, "instance %d: %s", i, why.c_str());
    if (params[i].precision != params[0].precision || params[i].device != params[0].device)
      return fail(nullptr, LBM_ERR_UNSUPPORTED, "all instances must share precision and device");
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0)
    return fail(nullptr, LBM_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  if (params[0].device < 0 || params[0].device >= ndev)
    return fail(nullptr, LBM_ERR_INVALID_ARG, "device %d out of range", params[0].device);
  lbm_t h = new lbm_s();
  h->device = params[0].device;
  DevGuard g(h->device);
  h->precision = params[0].precision;
  h->esize = h->precision == LBM_FP32 ? 4 : 2;
  h->stats_every = params[0].stats_every;
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (params[0].stream) {
    h->stream = static_cast<cudaStream_t>(params[0].stream);
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      int rc = fail(nullptr, LBM_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
      release(h);
      return rc;
    }
    h->own_stream = true;
  }
  // graphs cannot be captured on the legacy default stream
  h->use_graphs = h->stream != nullptr && h->stream != cudaStreamLegacy;
  h->inst.resize(count);
  int rc = alloc_common(h);
  for (int i = 0; rc == LBM_OK && i < count; ++i) {
    Inst& I = h->inst[i];
    I.p = params[i];
    derive(I);
    I.f_bytes = (size_t)19 * I.p.nz * I.p.ny * I.nxp * h->esize;
    e = cudaMalloc(&I.f, I.f_bytes);
    if (e != cudaSuccess) {
      rc = fail(h, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                "population array of instance %d (%zu bytes): %s", i, I.f_bytes, cudaGetErrorString(e));
      break;
    }
    e = cudaMemsetAsync(I.f, 0, I.f_bytes, h->stream);
    if (e == cudaSuccess) {
      std::vector<float> tb = force_tables(I);
      e = cudaMalloc(&I.tables, sizeof(float) * tb.size());
      if (e == cudaSuccess)
        e = cudaMemcpy(I.tables, tb.data(), sizeof(float) * tb.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) rc = fail(h, LBM_ERR_CUDA, "setup of instance %d: %s", i, cudaGetErrorString(e));
  }
  if (rc == LBM_OK) rc = choose_config(h, params[0]);
  if (rc == LBM_OK) {
    // autotuning ran steps on the rest state: restore it and the clock
    for (Inst& I : h->inst) {
      e = cudaMemsetAsync(I.f, 0, I.f_bytes, h->stream);
      if (e != cudaSuccess) rc = fail(h, LBM_ERR_CUDA, "reset: %s", cudaGetErrorString(e));
    }
    h->t = 0;
  }
  if (rc == LBM_OK) {
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = fail(h, LBM_ERR_CUDA, "create: %s", cudaGetErrorString(e));
  }
  if (rc != LBM_OK) {
    g_create_error = h->err;
    release(h);
    return rc;
  }
  *out = h;
  return LBM_OK;
}

// ---- autotuner ------------------------------------------------------------------

struct Candidate {
  int kind, threads, stages, tile_bytes, rows, slot_bytes;
  int layout;  // 0 population-major, 1 row-interleaved
};

// TMA candidate with R x-lines per tile: the compile-time slot layout when
// the stage count has one and R x-lines of every instance fit a slot
// (row_stage = 19 x-lines of the widest instance), else the runtime stride.
Candidate tma_candidate(int64_t row_stage, int R, int stages, int threads, bool slots = true,
                        bool two_blocks = false) {
  const int64_t seg = row_stage / 19 * R;  // bytes of R x-lines of one population
  if (slots && two_blocks && stages == 2 && seg <= kSlot2h) return {2, threads, stages, 19 * kSlot2h, R, kSlot2h, 0};
  if (slots && !two_blocks && stages == 3 && seg <= kSlot3) return {2, threads, stages, 19 * kSlot3, R, kSlot3, 0};
  if (slots && !two_blocks && stages == 2 && seg <= kSlot2) return {2, threads, stages, 19 * kSlot2, R, kSlot2, 0};
  return {2, threads, stages, (int)((row_stage * R + 15) / 16 * 16), R, 0, 0};
}

int apply_candidate(lbm_t h, const Candidate& c) {
  h->kind = c.kind;
  h->threads = c.threads;
  h->stages = c.stages;
  h->tile_bytes_max = c.tile_bytes;
  h->rows_fixed = c.rows;
  h->slot_bytes = c.kind == 2 ? c.slot_bytes : 0;
  h->layout = c.layout;
  if (c.kind == 2) {
    int max_nx = 1;
    for (const Inst& I : h->inst) max_nx = std::max(max_nx, I.p.nx);
    h->smem = tma_smem_bytes(c.stages, c.tile_bytes, max_nx);
    if (tma_prepare(h->precision, h->smem) != cudaSuccess) return LBM_ERR_UNSUPPORTED;
    h->bps = tma_max_blocks_per_sm(h->precision, (h->slot_bytes == 0 && h->layout == 1) ? kSlotGrouped : h->slot_bytes,
                                   c.threads, h->smem);
  } else {
    h->smem = 0;
    h->bps = direct_max_blocks_per_sm(h->precision, c.threads);
  }
  if (h->bps < 1) return LBM_ERR_UNSUPPORTED;
  h->grid = h->num_sms * h->bps;
  return build_tiles(h);
}

// Largest stage the TMA kernel can use for every instance (one row of 19
// segments must fit), or 0 if some instance's row is too long.
int64_t max_row_stage_bytes(lbm_t h) {
  int64_t m = 0;
  for (const Inst& I : h->inst) m = std::max<int64_t>(m, (int64_t)19 * I.nxp * (int64_t)h->esize);
  return m;
}

double time_candidate(lbm_t h, int steps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const bool g = h->use_graphs;
  h->use_graphs = false;
  const int saved_every = h->stats_every;
  h->stats_every = 0;
  enqueue_steps(h, 0, 2);  // warm-up
  cudaEventRecord(a, h->stream);
  int rc = enqueue_steps(h, 0, steps);
  cudaEventRecord(b, h->stream);
  cudaError_t e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (rc == LBM_OK && e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  else ms = 1e30f;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->use_graphs = g;
  h->stats_every = saved_every;
  uint32_t err = 0;
  cudaMemcpy(&err, h->d_err, sizeof err, cudaMemcpyDeviceToHost);
  if (err) {
    cudaMemset(h->d_err, 0, sizeof err);
    return 1e30;
  }
  return ms;
}

int choose_config(lbm_t h, const lbm_params& p0) {
  const int requested_kind = p0.kernel, requested_rows = p0.tile_rows;
  std::vector<Candidate> cands;
  const int64_t row_stage = max_row_stage_bytes(h);
  const bool tma_ok = row_stage <= 110 * 1024;
  int max_nx = 1, min_ny = 1 << 30;
  for (const Inst& I : h->inst) {
    max_nx = std::max(max_nx, I.p.nx);
    min_ny = std::min(min_ny, I.p.ny);
  }
  // dynamic shared memory left beside the static reduction scratch of the stats variant
  const int64_t smem_cap = 220 * 1024;
  // shared memory of one SM (228 KB on sm_100 / sm_103; 1 KB of it reserved per block)
  constexpr int kSmemPerSm = 233472;
  auto fits = [&](int stages, int64_t tb) {
    return (int64_t)tma_smem_bytes(stages, (int)tb, max_nx) <= smem_cap;
  };
  // population layout: lbm_params.layout 1 / 2 fixes it (population-major /
  // row-interleaved); 0 lets the autotuner try both for the TMA kernel and
  // means population-major otherwise
  const int lay_req = p0.layout;
  const int lay_fixed = lay_req == 2 ? 1 : 0;
  // a fully specified configuration skips the autotuner
  if (requested_kind == 1 && requested_rows > 0 && p0.threads > 0)
    return apply_candidate(h, {1, p0.threads, 0, 0, requested_rows, 0, lay_fixed});
  const bool allow_slots = p0.tma_slots == 0;
  if (requested_kind == 2 && requested_rows > 0 && p0.threads > 0 && p0.stages > 0) {
    Candidate c = p0.tma_slots == 2
                      ? tma_candidate(row_stage, requested_rows, p0.stages, p0.threads, true, true)
                      : tma_candidate(row_stage, requested_rows, p0.stages, p0.threads, allow_slots);
    if (p0.tma_slots == 2 && c.slot_bytes != kSlot2h)
      return fail(h, LBM_ERR_UNSUPPORTED, "tma_slots = 2 needs two stages whose tile rows fit a %d-byte slot", kSlot2h);
    if (!fits(p0.stages, c.tile_bytes)) c = tma_candidate(row_stage, requested_rows, p0.stages, p0.threads, false);
    if (!tma_ok || !fits(p0.stages, c.tile_bytes))
      return fail(h, LBM_ERR_UNSUPPORTED, "requested TMA stages do not fit shared memory");
    c.layout = lay_fixed;
    return apply_candidate(h, c);
  }
  if (requested_kind == 1 || requested_kind == 0)
    cands.push_back({1, 256, 0, 0, requested_rows, 0, lay_fixed});
  if ((requested_kind == 2 || requested_kind == 0) && tma_ok) {
    // a stage holds R x-lines of every population (exact multiples of one row stage)
    const int row_opts[] = {1, 2, 3, 4, 6, 8, 12, 16};
    const int stage_opts[] = {2, 3, 4};
    const int thread_opts[] = {256, 384, 512};
    for (int R : row_opts) {
      if (requested_rows > 0 && R != requested_rows) continue;
      if (R > 1 && R > min_ny) break;
      if ((row_stage * R + 15) / 16 * 16 > 96 * 1024) break;
      for (int s : stage_opts) {
        for (int th : thread_opts) {
          Candidate c = tma_candidate(row_stage, R, s, th, allow_slots);
          if (!fits(s, c.tile_bytes)) c = tma_candidate(row_stage, R, s, th, false);
          if (!fits(s, c.tile_bytes)) continue;
          for (int lay = 0; lay < 2; ++lay) {
            if ((lay_req == 1 && lay == 1) || (lay_req == 2 && lay == 0)) continue;
            c.layout = lay;
            cands.push_back(c);
            // row-interleaved one-x-line tiles also in the runtime stride, where
            // an odd step moves each slot group of a cell row in one copy
            if (lay == 1 && R == 1 && c.slot_bytes != 0) {
              Candidate r = tma_candidate(row_stage, R, s, th, false);
              r.layout = 1;
              if (fits(s, r.tile_bytes)) cands.push_back(r);
            }

          }
        }
      }
    }
    // two co-resident blocks of 256 threads per SM: stages small enough for a
    // second block, so that one block's pipeline fill and drain overlap the
    // other's steady state (small lattices, where each block sees few tiles
    // per step): the largest tiles that fit, and the listed smaller ones, in
    // the runtime stride and, with two stages, in kSlot2h slots
    // (population-major array; the row-interleaved one only for one-x-line tiles)
    for (int s : {2, 3}) {
      const int64_t per_block = kSmemPerSm / 2 - 1024 - tma_smem_bytes(s, 0, max_nx);
      const int rmax = (int)std::min<int64_t>(per_block / (s * row_stage), std::max(1, min_ny));
      if (rmax < 1) continue;
      std::vector<int> rs_two = {rmax};
      for (int R : row_opts)
        if (R < rmax) rs_two.push_back(R);
      for (int R : rs_two) {
        if (requested_rows > 0 && R != requested_rows) continue;
        for (bool slot_variant : {false, true}) {
          if (slot_variant && (s != 2 || !allow_slots)) continue;
          Candidate c = tma_candidate(row_stage, R, s, 256, slot_variant, true);
          if (slot_variant && c.slot_bytes != kSlot2h) continue;
          if (2 * (tma_smem_bytes(s, c.tile_bytes, max_nx) + 1024) > kSmemPerSm) continue;
          for (int lay = 0; lay < 2; ++lay) {
            if ((lay_req == 1 && lay == 1) || (lay_req == 2 && lay == 0)) continue;
            if (lay == 1 && R > 1) continue;
            c.layout = lay;
            cands.push_back(c);
          }
        }
      }
    }
    if (requested_kind == 2 && cands.empty() && fits(2, (row_stage + 15) / 16 * 16)) {
      Candidate c = tma_candidate(row_stage, 1, 2, 256, allow_slots);
      c.layout = lay_fixed;
      cands.push_back(c);
    }
  }
  if (cands.empty())
    return fail(h, LBM_ERR_UNSUPPORTED, "no kernel configuration fits this lattice");
  if (cands.size() == 1) return apply_candidate(h, cands[0]);
  // time each candidate on the rest state
  int64_t cells = 0;
  for (const Inst& I : h->inst) cells += I.ncell;
  const int steps = cells > (int64_t)64 << 20 ? 2 : (cells > (int64_t)4 << 20 ? 4 : 8);
  double best = 1e300;
  Candidate bc = cands[0];
  for (const Candidate& c : cands) {
    if (apply_candidate(h, c) != LBM_OK) continue;
    const double ms = time_candidate(h, steps);
    if (ms < best) {
      best = ms;
      bc = c;
    }
  }
  return apply_candidate(h, bc);
}

}  // namespace

namespace lbm {
// Error text for entry points that take no handle (read by lbm_last_error(NULL)).
void set_global_error(const char* msg) { g_create_error = msg; }
}  // namespace lbm

// ---- public entry points ------------------------------------------------------------

LBM_API int lbm_create(const lbm_params* params, lbm_t* out) { return create_impl(params, 1, out); }

LBM_API int lbm_create_batch(const lbm_params* params, int32_t count, lbm_t* out) {
  return create_impl(params, count, out);
}

LBM_API int lbm_batch_create(const lbm_params* params, int32_t count, lbm_t* out) {
  return create_impl(params, count, out);
}

LBM_API int lbm_destroy(lbm_t h) {
  if (!h) return LBM_OK;
  DevGuard g(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  release(h);
  return LBM_OK;
}

LBM_API int lbm_count(lbm_t h) { return h ? (int)h->inst.size() : 0; }

#define CHECK_INST(h, i)                                                              \
  do {                                                                                \
    if (!(h)) return fail(nullptr, LBM_ERR_INVALID_ARG, "null handle");               \
    if ((i) < 0 || (i) >= (int)(h)->inst.size())                                      \
      return fail((h), LBM_ERR_INVALID_ARG, "instance %d out of range", (int)(i));    \
  } while (0)

namespace {

// A handle with one instance restarts its clock at an initialisation (which
// changes the state: every caller of reset_time initialises).
int reset_time(lbm_t h) {
  ++h->version;
  if (h->inst.size() == 1 && h->t != 0) {
    h->t = 0;
    h->rec_steps.clear();
    h->inst[0].rec_read = 0;
    CK(h, cudaMemsetAsync(h->d_seq, 0, 2 * sizeof(unsigned long long), h->stream));
  }
  return LBM_OK;
}

// Equilibrium of a given FP64 or FP32 velocity for cells [c0, c0 + n).
cudaError_t init_from(const InstDesc& d, int precision, bool odd, const double* u, int64_t ustride,
                      int64_t c0, int64_t n, cudaStream_t st) {
  return launch_init(d, precision, odd, 3, 0.0, u, ustride, c0, n, st);
}
cudaError_t init_from(const InstDesc& d, int precision, bool odd, const float* u, int64_t ustride,
                      int64_t c0, int64_t n, cudaStream_t st) {
  return launch_init(d, precision, odd, u, ustride, c0, n, st);
}

// Local equilibrium of a given velocity field u[3][nz][ny][nx] of type U (FP64
// or FP32) in host memory (where = 0, staged copies), device memory (1) or
// page-locked host memory read in place (2).
template <typename U>
int init_velocity(lbm_t h, int32_t inst, const U* u, int32_t where) {
  Inst& I = h->inst[inst];
  const InstDesc& d = h->h_desc[inst];
  const bool odd = (h->t & 1) != 0;
  if (where == 1) {
    CK(h, init_from(d, h->precision, odd, u, I.ncell, 0, I.ncell, h->stream));
  } else if (where == 2) {
    // both ends of the 3 ncell values must be page-locked memory the device can address
    const U* ends[2] = {u, u + 3 * I.ncell - 1};
    const U* dev_u = nullptr;
    const bool pending = cudaPeekAtLastError() != cudaSuccess;  // the caller's, left alone
    for (int e = 0; e < 2; ++e) {
      cudaPointerAttributes at{};
      const cudaError_t ae = cudaPointerGetAttributes(&at, ends[e]);
      if (ae != cudaSuccess || at.type != cudaMemoryTypeHost || !at.devicePointer) {
        if (ae != cudaSuccess && !pending) (void)cudaGetLastError();  // this lookup's own failure
        return fail(h, LBM_ERR_INVALID_ARG, "u_on_device = 2 needs page-locked host memory");
      }
      if (e == 0) dev_u = static_cast<const U*>(at.devicePointer);
    }
    CK(h, init_from(d, h->precision, odd, dev_u, I.ncell, 0, I.ncell, h->stream));
  } else if (where == 0) {
    const int64_t chunk = std::min<int64_t>(I.ncell, kChunkCells);
    int rc = ensure_scratch(h, sizeof(U) * 3 * (size_t)chunk);
    if (rc != LBM_OK) return rc;
    U* s = static_cast<U*>(h->d_scratch);
    for (int64_t c0 = 0; c0 < I.ncell; c0 += chunk) {
      const int64_t n = std::min(chunk, I.ncell - c0);
      for (int dcomp = 0; dcomp < 3; ++dcomp)
        CK(h, cudaMemcpyAsync(s + dcomp * n, u + dcomp * I.ncell + c0, sizeof(U) * n,
                              cudaMemcpyHostToDevice, h->stream));
      CK(h, init_from(d, h->precision, odd, s, n, c0, n, h->stream));
    }
  } else {
    return fail(h, LBM_ERR_INVALID_ARG, "u_on_device must be 0, 1 or 2");
  }
  return LBM_OK;
}

}  // namespace

LBM_API int lbm_init_field(lbm_t h, int32_t inst, int32_t mode, double amplitude, const double* u,
                           int32_t u_on_device) {
  CHECK_INST(h, inst);
  DevGuard g(h->device);
  if (mode < LBM_INIT_REST || mode > LBM_INIT_VELOCITY)
    return fail(h, LBM_ERR_INVALID_ARG, "unknown init mode %d", mode);
  if (mode == LBM_INIT_VELOCITY && !u) return fail(h, LBM_ERR_INVALID_ARG, "velocity pointer is null");
  if (!std::isfinite(amplitude)) return fail(h, LBM_ERR_INVALID_ARG, "non-finite amplitude");
  if (mode == LBM_INIT_VELOCITY && (u_on_device < 0 || u_on_device > 2))
    return fail(h, LBM_ERR_INVALID_ARG, "u_on_device must be 0, 1 or 2");
  int rc = reset_time(h);
  if (rc != LBM_OK) return rc;
  if (mode == LBM_INIT_VELOCITY) return init_velocity<double>(h, inst, u, u_on_device);
  const Inst& I = h->inst[inst];
  CK(h, launch_init(h->h_desc[inst], h->precision, (h->t & 1) != 0, mode, amplitude,
                    nullptr, 0, 0, I.ncell, h->stream));
  return LBM_OK;
}

LBM_API int lbm_init_random_spectrum(lbm_t h, int32_t inst, uint64_t seed, double urms, double k0,
                                     float* u_out, int32_t u_out_on_device) {
  CHECK_INST(h, inst);
  DevGuard g(h->device);
  const Inst& I = h->inst[inst];
  const lbm_params& p = I.p;
  if (!(urms > 0.0) || !std::isfinite(urms)) return fail(h, LBM_ERR_INVALID_ARG, "urms must be finite and > 0");
  if (!(k0 > 0.0) || !std::isfinite(k0)) return fail(h, LBM_ERR_INVALID_ARG, "k0 must be finite and > 0");
  if (p.nx < 4 || p.ny < 4 || p.nz < 4)
    return fail(h, LBM_ERR_INVALID_ARG, "the random field needs every extent >= 4");
  if (u_out && (u_out_on_device < 0 || u_out_on_device > 1))
    return fail(h, LBM_ERR_INVALID_ARG, "u_out_on_device must be 0 or 1");
  int rc = reset_time(h);
  if (rc != LBM_OK) return rc;
  float* u = nullptr;
  cudaError_t e = cudaMalloc(&u, sizeof(float) * 3 * (size_t)I.ncell);
  if (e != cudaSuccess)
    return fail(h, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "velocity buffer: %s",
                cudaGetErrorString(e));
  cudaError_t ce = cudaSuccess;
  const char* what = random_velocity_f32(p.nx, p.ny, p.nz, seed, urms, k0, u, h->stream, &ce);
  if (what) {
    cudaFree(u);
    return fail(h, ce == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "random field: %s: %s", what,
                cudaGetErrorString(ce));
  }
  e = init_from(h->h_desc[inst], h->precision, (h->t & 1) != 0, (const float*)u, I.ncell, 0, I.ncell, h->stream);
  if (e == cudaSuccess && u_out)
    e = cudaMemcpyAsync(u_out, u, sizeof(float) * 3 * (size_t)I.ncell,
                        u_out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
  const cudaError_t se = cudaStreamSynchronize(h->stream);
  cudaFree(u);
  if (e != cudaSuccess) return fail(h, LBM_ERR_CUDA, "random-field initialisation: %s", cudaGetErrorString(e));
  if (se != cudaSuccess) return fail(h, LBM_ERR_CUDA, "random-field initialisation: %s", cudaGetErrorString(se));
  return LBM_OK;
}

LBM_API int lbm_init_velocity_f32(lbm_t h, int32_t inst, const float* u, int32_t u_on_device) {
  CHECK_INST(h, inst);
  DevGuard g(h->device);
  if (!u) return fail(h, LBM_ERR_INVALID_ARG, "velocity pointer is null");
  if (u_on_device < 0 || u_on_device > 2) return fail(h, LBM_ERR_INVALID_ARG, "u_on_device must be 0, 1 or 2");
  int rc = reset_time(h);
  if (rc != LBM_OK) return rc;
  return init_velocity<float>(h, inst, u, u_on_device);
}

LBM_API int lbm_step(lbm_t h, int64_t n) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "null handle");
  if (n < 0) return fail(h, LBM_ERR_INVALID_ARG, "n < 0");
  DevGuard g(h->device);
  return run_steps(h, n);
}

LBM_API int lbm_batch_step(lbm_t h, int64_t n) { return lbm_step(h, n); }

LBM_API int lbm_sync(lbm_t h) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "null handle");
  DevGuard g(h->device);
  return check_err(h);
}

LBM_API int64_t lbm_time(lbm_t h) { return h ? h->t : -1; }

LBM_API int lbm_stats(lbm_t h, int32_t inst, int32_t what, lbm_stats_t* out) {
  CHECK_INST(h, inst);
  if (!out) return fail(h, LBM_ERR_INVALID_ARG, "null output");
  DevGuard g(h->device);
  Inst& I = h->inst[inst];
  const bool need_u = (what & (LBM_STATS_SPECTRUM | LBM_STATS_STRUCTURE)) != 0;
  int rc = diag_pass(h, inst, need_u, false, -1, 0, true);
  if (rc != LBM_OK) return rc;
  std::vector<double> r(kNP);
  CK(h, cudaMemcpyAsync(r.data(), h->d_results + (size_t)inst * kNP, sizeof(double) * kNP,
                        cudaMemcpyDeviceToHost, h->stream));
  std::vector<uint32_t> hist(I.hist_bins + 1);
  CK(h, cudaMemcpyAsync(hist.data(), I.hist, sizeof(uint32_t) * hist.size(), cudaMemcpyDeviceToHost,
                        h->stream));
  rc = check_err(h);
  if (rc != LBM_OK) return rc;
  std::memset(out, 0, sizeof *out);
  fill_from_sums(out, r.data(), I, h->t);
  // percentiles: centre of the first bin whose cumulative count reaches p n
  const double pct[4] = {0.05, 0.50, 0.95, 0.99};
  double* dst[4] = {&out->theta_p05, &out->theta_p50, &out->theta_p95, &out->theta_p99};
  const double width = I.hist_max / I.hist_bins;
  for (int q = 0; q < 4; ++q) {
    const double target = pct[q] * (double)out->cells;
    double cum = 0.0;
    int b = 0;
    for (; b < I.hist_bins; ++b) {
      cum += hist[b];
      if (cum >= target) break;
    }
    *dst[q] = b < I.hist_bins ? (b + 0.5) * width : I.hist_max;
  }
  const double nan = std::nan("");
  out->L = out->eps_spec = out->eta = out->lambda = out->u_rms = out->Re_lambda = nan;
  out->u_rms = std::sqrt(2.0 * out->E_k / 3.0);  // Eq. (rms_velocity)
  const lbm_params& p = I.p;
  if (what & LBM_STATS_SPECTRUM) {
    const int kmax = max_shell(p.nx, p.ny, p.nz);
    std::vector<double> E(kmax + 1);
    rc = spectrum_device(h, inst, kmax, E.data());
    if (rc != LBM_OK) return rc;
    // Eqs. (integral_length_scale) - (dissipation_rate) with k_s = 2 pi s / nx
    double sE = 0, sEk = 0, sk2E = 0;
    for (int s = 1; s <= kmax; ++s) {
      const double k = 2.0 * kPi * s / p.nx;
      sE += E[s];
      sEk += E[s] / k;
      sk2E += k * k * E[s];
    }
    out->L = 0.75 * kPi * sEk / sE;
    out->eps_spec = 2.0 * I.nu0 * sk2E;
    out->eta = std::pow(I.nu0 * I.nu0 * I.nu0 / out->eps_spec, 0.25);
    out->lambda = std::sqrt(15.0 * I.nu0 * out->u_rms * out->u_rms / out->eps_spec);
    out->Re_lambda = out->u_rms * out->lambda / I.nu0;  // Sec. 3.1
  }
  if (what & LBM_STATS_STRUCTURE) {
    std::vector<int> rs = separations(std::min({p.nx, p.ny, p.nz}));
    if ((int)rs.size() > LBM_MAX_R) rs.resize(LBM_MAX_R);
    out->nr = 0;
    if (rs.empty()) return LBM_OK;
    const int blocks = std::min(2 * h->num_sms, 1024);
    const size_t need = ((size_t)blocks + 1) * 6 * rs.size();
    if (need > h->spec_elems) {
      if (h->d_spec) cudaFree(h->d_spec);
      h->d_spec = nullptr;
      CK(h, cudaMalloc(&h->d_spec, need * sizeof(double)));
      h->spec_elems = need;
    }
    out->nr = (int)rs.size();
    // every separation in one launch into a [blocks][nr x 6] table, one column
    // sum, one read-back
    const int cols = 6 * (int)rs.size();
    CK(h, launch_struct_multi(I.u, p.nx, p.ny, p.nz, rs.data(), (int)rs.size(), h->d_spec, blocks, h->stream));
    CK(h, launch_sum_cols(h->d_spec, blocks, cols, h->d_spec + (size_t)blocks * cols, h->stream));
    std::vector<double> sp(cols);
    CK(h, cudaMemcpyAsync(sp.data(), h->d_spec + (size_t)blocks * cols, sizeof(double) * cols,
                          cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (size_t k = 0; k < rs.size(); ++k) {
      out->r[k] = rs[k];
      for (int q = 0; q < 6; ++q) out->Sp[k][q] = sp[6 * k + q] / (3.0 * (double)I.ncell);
      out->F4[k] = out->Sp[k][3] / (out->Sp[k][1] * out->Sp[k][1]);  // Eq. (flatness)
    }
  }
  return LBM_OK;
}

LBM_API int lbm_batch_stats(lbm_t h, int32_t what, lbm_stats_t* out) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "null handle");
  if (!out) return fail(h, LBM_ERR_INVALID_ARG, "null output");
  for (int i = 0; i < (int)h->inst.size(); ++i) {
    const int rc = lbm_stats(h, i, what, out + i);
    if (rc != LBM_OK) return rc;
  }
  return LBM_OK;
}

LBM_API int lbm_series(lbm_t h, int32_t inst, lbm_record_t* out, int32_t max, int32_t* count) {
  CHECK_INST(h, inst);
  if (!count || (max > 0 && !out)) return fail(h, LBM_ERR_INVALID_ARG, "null output");
  DevGuard g(h->device);
  *count = 0;
  unsigned long long seq = 0;
  CK(h, cudaMemcpyAsync(&seq, h->d_seq, sizeof seq, cudaMemcpyDeviceToHost, h->stream));
  int rc = check_err(h);
  if (rc != LBM_OK) return rc;
  Inst& I = h->inst[inst];
  uint64_t first = I.rec_read;
  if (seq > (unsigned long long)kRingCap && first < seq - kRingCap) first = seq - kRingCap;
  const int ninst = (int)h->inst.size();
  std::vector<double> r(kNP);
  for (uint64_t k = first; k < seq && *count < max; ++k) {
    CK(h, cudaMemcpy(r.data(), h->d_ring + ((k % kRingCap) * ninst + inst) * kNP,
                     sizeof(double) * kNP, cudaMemcpyDeviceToHost));
    lbm_stats_t s;
    fill_from_sums(&s, r.data(), I, k < h->rec_steps.size() ? h->rec_steps[k] : -1);
    lbm_record_t& o = out[*count];
    o.step = s.step;
    o.mass = s.mass;
    for (int q = 0; q < 3; ++q) o.momentum[q] = s.momentum[q];
    o.E_k = s.E_k;
    o.inj = s.inj;
    o.eps0 = s.eps0;
    o.eps_sgs = s.eps_sgs;
    o.theta_mean = s.theta_mean;
    o.theta_var = s.theta_var;
    o.theta_min = s.theta_min;
    o.theta_max = s.theta_max;
    ++*count;
    I.rec_read = k + 1;
  }
  return LBM_OK;
}

LBM_API int lbm_energy_balance(const lbm_record_t* rec, int32_t n, double* residual, int64_t* at) {
  if (!rec || !residual || n < 3)
    return fail(nullptr, LBM_ERR_INVALID_ARG, "energy balance needs >= 3 records and outputs");
  for (int k = 1; k < n; ++k)
    if (rec[k].step <= rec[k - 1].step)
      return fail(nullptr, LBM_ERR_INVALID_ARG, "record times must increase");
  for (int k = 1; k + 1 < n; ++k) {
    // Eq. (energy_balance): eps = -dE_k/dt + <F.u>, central difference in time
    const double dEdt = (rec[k + 1].E_k - rec[k - 1].E_k) / (double)(rec[k + 1].step - rec[k - 1].step);
    const double eps = rec[k].eps0 + rec[k].eps_sgs;
    residual[k - 1] = (eps - (-dEdt + rec[k].inj)) / eps;
    if (at) at[k - 1] = rec[k].step;
  }
  return LBM_OK;
}

LBM_API int lbm_spectrum(lbm_t h, int32_t inst, double* E, int32_t kmax) {
  CHECK_INST(h, inst);
  if (!E || kmax < 0) return fail(h, LBM_ERR_INVALID_ARG, "null output or kmax < 0");
  DevGuard g(h->device);
  const lbm_params& p = h->inst[inst].p;
  const int smax = max_shell(p.nx, p.ny, p.nz);  // shells beyond hold no mode
  for (int s = smax + 1; s <= kmax; ++s) E[s] = 0.0;
  int rc = LBM_OK;
  if (h->inst[inst].u_version != h->version) {  // the velocity of this state is not at hand
    rc = diag_pass(h, inst, true, false, -1, 0, false);
    if (rc != LBM_OK) return rc;
  }
  rc = spectrum_device(h, inst, std::min(kmax, smax), E);
  if (rc != LBM_OK) return rc;
  return check_err(h);
}

LBM_API int lbm_histogram(lbm_t h, int32_t inst, uint64_t* counts, int32_t bins) {
  CHECK_INST(h, inst);
  Inst& I = h->inst[inst];
  if (!counts || bins != I.hist_bins) return fail(h, LBM_ERR_INVALID_ARG, "bins must equal hist_bins (%d)", I.hist_bins);
  if (!I.hist) return fail(h, LBM_ERR_INVALID_ARG, "no histogram yet: call lbm_stats first");
  DevGuard g(h->device);
  std::vector<uint32_t> hist(I.hist_bins + 1);
  CK(h, cudaMemcpyAsync(hist.data(), I.hist, sizeof(uint32_t) * hist.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  for (size_t b = 0; b < hist.size(); ++b) counts[b] = hist[b];
  return LBM_OK;
}

LBM_API int lbm_get_populations(lbm_t h, int32_t inst, double* host, int32_t shifted) {
  CHECK_INST(h, inst);
  if (!host) return fail(h, LBM_ERR_INVALID_ARG, "null output");
  DevGuard g(h->device);
  Inst& I = h->inst[inst];
  const int64_t chunk = std::min<int64_t>(I.ncell, kChunkCells);
  int rc = ensure_scratch(h, sizeof(double) * (size_t)chunk);
  if (rc != LBM_OK) return rc;
  double* s = static_cast<double*>(h->d_scratch);
  const bool odd = (h->t & 1) != 0;
  for (int a = 0; a < 19; ++a)
    for (int64_t c0 = 0; c0 < I.ncell; c0 += chunk) {
      const int64_t n = std::min(chunk, I.ncell - c0);
      CK(h, launch_get_pop(h->h_desc[inst], h->precision, odd, a, s, shifted, c0, n, h->stream));
      CK(h, cudaMemcpyAsync(host + a * I.ncell + c0, s, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    }
  CK(h, cudaStreamSynchronize(h->stream));
  return check_err(h);
}

LBM_API int lbm_set_populations(lbm_t h, int32_t inst, const double* host, int32_t shifted) {
  CHECK_INST(h, inst);
  if (!host) return fail(h, LBM_ERR_INVALID_ARG, "null input");
  DevGuard g(h->device);
  ++h->version;
  Inst& I = h->inst[inst];
  const int64_t chunk = std::min<int64_t>(I.ncell, kChunkCells);
  int rc = ensure_scratch(h, sizeof(double) * (size_t)chunk);
  if (rc != LBM_OK) return rc;
  double* s = static_cast<double*>(h->d_scratch);
  const bool odd = (h->t & 1) != 0;
  for (int a = 0; a < 19; ++a)
    for (int64_t c0 = 0; c0 < I.ncell; c0 += chunk) {
      const int64_t n = std::min(chunk, I.ncell - c0);
      CK(h, cudaMemcpyAsync(s, host + a * I.ncell + c0, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
      CK(h, launch_set_pop(h->h_desc[inst], h->precision, odd, a, s, shifted, c0, n, h->stream));
    }
  CK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

LBM_API int lbm_set_time(lbm_t h, int64_t t) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "null handle");
  if (t < 0) return fail(h, LBM_ERR_INVALID_ARG, "t < 0");
  DevGuard g(h->device);
  ++h->version;
  if ((t & 1) != (h->t & 1)) {
    size_t plane = 0;
    for (const Inst& I : h->inst) plane = std::max(plane, (size_t)I.p.nz * I.p.ny * I.nxp * h->esize);
    int rc = ensure_scratch(h, 2 * plane);
    if (rc != LBM_OK) return rc;
    const bool from_odd = (h->t & 1) != 0;
    for (size_t i = 0; i < h->inst.size(); ++i)
      for (int a = 0; a < 18; a += 2)
        CK(h, launch_relayout_pair(h->h_desc[i], h->precision, from_odd, a, h->d_scratch, h->stream));
  }
  h->t = t;
  CK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

LBM_API int lbm_get_fields(lbm_t h, int32_t inst, double* drho, double* u, double* snorm,
                           double* theta) {
  CHECK_INST(h, inst);
  DevGuard g(h->device);
  Inst& I = h->inst[inst];
  int rc = diag_pass(h, inst, u != nullptr, drho || snorm || theta, -1, 0, false);
  if (rc != LBM_OK) return rc;
  std::vector<float> buf;
  auto fetch = [&](const float* src, double* dst, int64_t n) -> int {
    buf.resize((size_t)n);
    CK(h, cudaMemcpyAsync(buf.data(), src, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int64_t k = 0; k < n; ++k) dst[k] = buf[k];
    return LBM_OK;
  };
  if (u && (rc = fetch(I.u, u, 3 * I.ncell)) != LBM_OK) return rc;
  if (drho && (rc = fetch(I.aux, drho, I.ncell)) != LBM_OK) return rc;
  if (snorm && (rc = fetch(I.aux + I.ncell, snorm, I.ncell)) != LBM_OK) return rc;
  if (theta && (rc = fetch(I.aux + 2 * I.ncell, theta, I.ncell)) != LBM_OK) return rc;
  return check_err(h);
}

LBM_API int lbm_get_velocity(lbm_t h, int32_t inst, double* u) {
  CHECK_INST(h, inst);
  if (!u) return fail(h, LBM_ERR_INVALID_ARG, "null output");
  return lbm_get_fields(h, inst, nullptr, u, nullptr, nullptr);
}

LBM_API int lbm_get_theta_slice(lbm_t h, int32_t inst, int32_t axis, int32_t index, double* host) {
  CHECK_INST(h, inst);
  Inst& I = h->inst[inst];
  const lbm_params& p = I.p;
  const int ext[3] = {p.nx, p.ny, p.nz};
  if (axis < 0 || axis > 2 || index < 0 || index >= ext[axis] || !host)
    return fail(h, LBM_ERR_INVALID_ARG, "bad slice axis/index or null output");
  DevGuard g(h->device);
  int rc = diag_pass(h, inst, false, false, axis, index, false);
  if (rc != LBM_OK) return rc;
  const size_t n = axis == 0 ? (size_t)p.nz * p.ny : (axis == 1 ? (size_t)p.nz * p.nx : (size_t)p.ny * p.nx);
  std::vector<float> buf(n);
  CK(h, cudaMemcpyAsync(buf.data(), I.plane, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  for (size_t k = 0; k < n; ++k) host[k] = buf[k];
  return check_err(h);
}

LBM_API int lbm_device_ptr(lbm_t h, int32_t inst, void** ptr, size_t* bytes, int32_t* nxp) {
  CHECK_INST(h, inst);
  if (ptr) *ptr = h->inst[inst].f;
  if (bytes) *bytes = h->inst[inst].f_bytes;
  if (nxp) *nxp = h->inst[inst].nxp;
  return LBM_OK;
}

LBM_API int lbm_get_params(lbm_t h, int32_t inst, double* nu0, double* s_nu0, double* f0, double* C) {
  CHECK_INST(h, inst);
  const Inst& I = h->inst[inst];
  if (nu0) *nu0 = I.nu0;
  if (s_nu0) *s_nu0 = I.s_nu0;
  if (f0) *f0 = I.F0;
  if (C) *C = I.C;
  return LBM_OK;
}

LBM_API int lbm_kernel_config(lbm_t h, int32_t* kind, int32_t* tile_rows, int32_t* stages,
                              int32_t* threads, int32_t* blocks_per_sm, int32_t* layout,
                              int32_t* slot_bytes) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "null handle");
  if (kind) *kind = h->kind;
  if (tile_rows) *tile_rows = h->inst.empty() ? 0 : h->inst[0].rows;
  if (stages) *stages = h->stages;
  if (threads) *threads = h->threads;
  if (blocks_per_sm) *blocks_per_sm = h->bps;
  if (layout) *layout = h->layout == 1 ? 2 : 1;
  if (slot_bytes) *slot_bytes = h->kind == 2 ? h->slot_bytes : 0;
  return LBM_OK;
}

LBM_API int lbm_debug_withhold_load(lbm_t h, double wait_seconds) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "null handle");
  if (h->kind != 2) return fail(h, LBM_ERR_UNSUPPORTED, "the handle does not run the TMA kernel");
  if (!(wait_seconds > 0.0) || wait_seconds > 10.0)
    return fail(h, LBM_ERR_INVALID_ARG, "wait_seconds must be in (0, 10]");
  h->inject_withhold = 1;
  h->inject_wait_ns = (long long)(wait_seconds * 1e9);
  return LBM_OK;
}

LBM_API const char* lbm_last_error(lbm_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

LBM_API const char* lbm_version(void) { return "gb300-lbm 0.1 (sm_103a)"; }
