// Internal structures shared by the host side and the kernels of the GB300
// lattice Boltzmann library (not part of the public ABI, see include/lbm.h).
#pragma once

#include <cstdint>

namespace lbm {

// Per-instance description read by every kernel (device memory table).
struct InstDesc {
  void* f;                 // populations, storage type; value (a, x, y, z) at
                           // a slot_stride + z plane_stride + y row_stride + x
  const float* fx_of_y;    // Fx(y) table [ny]   (Eq. forcing_pattern)
  const float* fy_of_z;    // Fy(z) table [nz]
  const float* fz_of_x;    // Fz(x) table [nx]
  float fconst[3];         // uniform part of the force
  float nu0;               // bare viscosity
  float s_nu0;             // bare shear rate 1/(1/2 + 3 nu0)
  float C;                 // Smagorinsky constant
  int32_t strain_mode;     // 0: s9 = bare s_nu0 in the strain; 1: self-consistent s_nu(|S|)
  int32_t nx, ny, nz, nxp; // nxp: x stride (nx rounded up to the row alignment)
  int32_t row_copy_bytes;  // bytes of one x-line a bulk copy moves (nx cells, 16-byte multiple)
  // Population layout (elements): population-major [19][nz][ny][nxp]
  // (slot_stride = nz ny nxp, row_stride = nxp, slots in index order) or
  // row-interleaved [nz][ny][19][nxp] (slot_stride = nxp, row_stride = 19 nxp,
  // slot a at position gpos(a) of its cell row: slot_grouped = 1).
  int64_t slot_stride, plane_stride, row_stride;
  int32_t slot_grouped;
  int32_t rows;            // rows (y lines of nx cells) per tile
  int32_t tiles_per_plane; // ceil(ny / rows)
  int64_t tile_begin;      // first global tile of the instance
  int64_t tile_end;        // one past the last
  int64_t f_elems;         // storage elements of the population array (bounds checks)
};

// Outputs of the read-only statistics pass (single instance).
struct DiagOut {
  float* u;                // [3][nz][ny][nx] or null
  float* aux;              // [3][nz][ny][nx]: drho, |S|, theta, or null
  float* plane;            // theta plane or null
  int32_t plane_axis, plane_index;
  uint32_t* hist;          // [hist_bins + 1] or null
  int32_t hist_bins;
  float hist_scale;        // hist_bins / hist_max
};

// Number of doubles per block partial of the fused statistics.
constexpr int kNP = 20;
// Partial layout: 0 drho, 1..3 rho u, 4 u.u, 5 F.u, 6 |S|^2, 7 nu_t |S|^2,
// 8 theta, 9 theta^2, 10..15 ux ux, uy uy, uz uz, ux uy, ux uz, uy uz,
// 16 min theta, 17 max theta, 18 non-finite cells, 19 cells.
enum {
  P_DRHO = 0, P_MX, P_MY, P_MZ, P_UU, P_FU, P_SS, P_NUTSS, P_TH, P_TH2,
  P_XX, P_YY, P_ZZ, P_XY, P_XZ, P_YZ, P_THMIN, P_THMAX, P_BAD, P_CELLS
};
constexpr int kNSum = 16;

// Where a statistics-fused step writes its block partials.
struct StatsArgs {
  double* partials;        // [ninst][grid][kNP] (zeroed before the launch)
  int32_t grid;            // gridDim.x of the launch
};

// Error bits of the device error word.
constexpr uint32_t ERR_NONFINITE = 1u;
constexpr uint32_t ERR_TIMEOUT = 2u;
// After a timeout, loads already issued had not landed within the drain bound
// (kDrainRounds x wait_ns) when the block left.
constexpr uint32_t ERR_DRAIN = 4u;
// The checked build (-DLBM_BOUNDS_CHECK) found an index outside its buffer.
constexpr uint32_t ERR_BOUNDS = 8u;

// Step kernel modes.
enum { MODE_STEP = 0, MODE_STEP_STATS = 1, MODE_DIAG = 2 };

}  // namespace lbm
