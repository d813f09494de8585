// Host-side context of the QED particle-step library and the launch
// interfaces shared by its translation units.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/qed.h"
#include "qed_device.cuh"

namespace qed {

constexpr int kMaxPass = 64;        // nesting depth of products within one step
constexpr int kNumCounters = 22;    // device diagnostic counters
enum Counter {
  kCntEmissions = 0, kCntPairs, kCntSubLepton, kCntSubPhoton, kCntPmGt1, kCntPpGt1, kCntCapped,
  kCntAbsorbed, kCntOverflow, kCntNonfinite, kCntSpeciesSteps /* 4 slots: live particles per species */,
  kCntPhotonsMade = kCntSpeciesSteps + 4, kCntPairsMade, kCntThinned, kCntSchwinger, kCntSchwingerGt1,
  kCntBlockSteps,  // particle-steps advanced (and deposited) in cell-block order
  kCntTileDeposits // of those, deposits through the shared-memory tile of their cell block
};
constexpr int kWorkSlot = kMaxPass + 3;   // d_pend_count slot: work counter of the e-/e+/ion pass
constexpr int kEnsFieldStride = 8;        // per ensemble per step: E[3], B[3], |E|+|B|, pad
constexpr int kNsubKeys = 64;             // sort keys of the sub-interval estimate (last: >= 63)
constexpr int kMaxBins = 4096;
constexpr int kCompactTile = 2048;   // particles per tile of the compaction
constexpr int kBlockCells = 8;       // cell block edge (grid mode): 8 x 8 x 8 cells
constexpr int kBlockVolume = kBlockCells * kBlockCells * kBlockCells;

// n / d for n < 2^31 by a multiply-high and a shift (Granlund-Montgomery):
// fast_div_magic forms (m, l) for d on the host.
__device__ __forceinline__ unsigned fast_div(unsigned n, unsigned m, int l) { return (__umulhi(n, m) + n) >> l; }
inline void fast_div_magic(unsigned d, unsigned &m, int &l) {
  l = 0;
  while ((1ull << l) < d) ++l;
  m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
}
constexpr int kMaxStripes = 64;      // field update: stripes of the next step's mesh maxima
constexpr int kBlockChunk = 1024;    // records per work item of the cell-block kernel
// Current tile of a cell block (the deposit): the block plus a halo of H
// cells each side, kBlockCells + 2H + 1 nodes per axis.  The stencil of a
// move that starts in cell cs touches nodes cs - 1 .. cs + 2, so a tile of
// halo H takes every particle that starts within H - 1 cells of its block
// (H = 1: the block itself); H = 0 deposits without tiles (global atomics).
constexpr int kMaxDepositHalo = 4;
constexpr int kMaxTileNodes = kBlockCells + 2 * kMaxDepositHalo + 1;
__host__ __device__ constexpr int tile_nodes(int halo) { return kBlockCells + 2 * halo + 1; }

// One species store: a structure of arrays, double-buffered for compaction.
//   pos: {offset_x, offset_y, offset_z, weight}   (R4 = float4 or 2 x double2)
//   mom: {p_x, p_y, p_z, cell}   cell = linear lattice index, -1 when dead;
//        FP32 keeps the int bits in the 4th float, FP64 the value as a double
//   id : 64-bit particle id (keys the particle's random streams)
struct Store {
  void *pos[2] = {nullptr, nullptr};
  void *mom[2] = {nullptr, nullptr};
  uint64_t *id[2] = {nullptr, nullptr};
  int cur = 0;
  int64_t cap = 0;
};

// Everything the step kernel reads, passed by value.
template <typename R> struct StepArgs {
  // stores (current buffers), and the second position buffers (free between
  // compactions: the cell-block pass keeps its start points there)
  void *pos[4];
  void *mom[4];
  void *pos_scratch[4];
  uint64_t *id[4];
  long long *count;        // [4] store sizes (live + dead), appended atomically
  const long long *nstart; // [4] sizes at the start of the step
  long long cap[4];
  // products evolving within the step
  void *pend[2];
  unsigned long long *pend_count;  // [kMaxPass + 2]
  long long pend_cap;
  // lattice; cell / n0 and cell / (n0 n1) by multiply-shift (div_m, div_l)
  unsigned div_m[2];
  int div_l[2];
  int n[3];
  int periodic[3];
  R d[3], inv_d[3];
  R jscale[3];             // d / (dt dx dy dz) per axis: current density of a unit charge moved one cell
  double dd[3], x0[3];
  // fields
  int field_mode;
  double fp[16];
  // ensembles: ensemble = id >> ens_shift (ens_shift 64: all in ensemble 0);
  // products keep the parent's ens_mask bits; per-step fields of each ensemble
  int ens_shift;
  int n_ens;
  unsigned long long ens_mask;
  const double *ens_table;  // n_ens x QED_ENS_STRIDE
  R *ens_field;            // n_ens x kEnsFieldStride, written by k_step_constants
  double ens_hmax;         // bound of |E| + |B| over the ensembles
  // Yee mesh: per-step maxima of |Ex| .. |Bz| (bit patterns), and where the
  // photon split threshold of the next compaction goes
  unsigned long long *grid_max;
  double *eps_star_out;
  // pairs from the vacuum (Sec. V.B)
  int schwinger;
  R schwinger_w;
  // event generator of the emission (Sec. IV.F-G): 0 modified, 1 alternative, 2 standard
  int generator;
  const R *std_cdf, *std_lnw;
  // generator factors (Sec. VI): keep = 1/f_g, wf = f_g / N_g
  R emit_keep, emit_wf, pair_keep, pair_wf;
  int emit_ng, pair_ng;
  // work stealing of the e-/e+/ion pass: particles per grab (0 = grid-stride)
  long long chunk;
  unsigned long long *work_massive;
  const R *E[3];
  const R *B[3];
  R *J[3];
  int deposit;
  int deposit_halo;        // current tiles of the deposit: halo H (0 = global atomics only)
  int deposit_grab;        // cell blocks a deposit block claims at a time (1 .. 32)
  int refill_lanes;        // cell-block pass, e-/e+: refill a warp's idle lanes at this many (0: batches)
  // generator
  R dt, kappa;
  int nsub_max, emission_on, pairs_on, same_step, pm_strict;
  unsigned seed;
  R charge[4], mass[4], inv_mass[4];
  const R *tab;
  const double *chi_star;  // photons below this chi_g cannot pair (per context)
  // grid mode, cell-block sort: blocks per axis, and per species the first
  // record of every block (nblk + 1 entries; the last is the sorted count)
  int nb[3];
  int nblk;
  const unsigned *blk_start[4];
  unsigned *work;          // work-stealing counters of the cell-block kernels (zeroed per step):
                           // [0] e-/e+ items, [1] deposit, [4] ion items, [5] drifted records
                           // ([2..3]: kWorkSlot)
  unsigned long long *drift;   // records whose stencil left their block's tile: species << 62 | index
  long long drift_cap;
  void *step_const;        // per-step field constants (written by k_step_constants)
  void *clock;             // device clock {t, step}: read and advanced once per step
  double dt_d;             // the step in FP64 (advances the clock)
  // diagnostics
  unsigned long long *counters;
  double *spectrum, *spectrum_energy;
  int nbins;
  double lg_lo, lg_inv_span;
  int *status;
  unsigned *barrier;       // [2]: arrivals, generation
};

}  // namespace qed

struct qed_ctx {
  int device = 0;
  int prec = 32;
  qed_grid_desc grid{};
  qed_species_desc species{};
  qed_params par{};
  qed::Store st[4];
  long long *d_count = nullptr;       // [4]
  long long *d_nstart = nullptr;      // [4]
  void *pend[2] = {nullptr, nullptr};
  long long pend_cap = 0;
  unsigned long long *d_pend_count = nullptr;
  unsigned long long *d_counters = nullptr;
  double *d_spec = nullptr, *d_spec_e = nullptr;
  int *d_status = nullptr;
  unsigned *d_barrier = nullptr;
  void *d_tables = nullptr;
  double *d_chi_star = nullptr;       // pair-skip threshold derived from the tables
  double *d_eps_star = nullptr;       // photons below this |p| cannot pair in the analytic field
  void *d_step_const = nullptr;       // per-step field constants
  double *d_ens = nullptr;            // ensemble table (2^ens_bits rows)
  float *d_ens_h = nullptr;           // per ensemble |E0| + |Eu| + |Bu| (sort key)
  void *d_ens_field = nullptr;        // per-step ensemble fields (context precision)
  int n_ens = 0;
  int ens_cap = 0;                    // rows allocated
  double ens_hmax = 0.0;
  int key_ensembles = 0;              // ensembles: sort keys are estimated sub-interval counts
  double last_dt = 0.0;               // dt of the latest qed_step (the sort key uses it)
  int ext = 0;                        // ensembles or generator factors: EXT kernels
  void *d_thin = nullptr;             // thinning: per group count, weight, survivors' weight
  unsigned long long *d_grid_max = nullptr;   // Yee mesh: |E|, |B| component maxima per step
  unsigned long long *d_drift = nullptr;      // deposit: the records that left their block's tile
  long long drift_cap = 0;
  unsigned long long *d_grid_max_next = nullptr;  // [kMaxStripes][6]: the same, of the fields the last update wrote
  int grid_max_ready = 0;             // d_grid_max_next holds the maxima of the current fields
  void *d_std_cdf = nullptr;          // standard generator: kStdRows x kStdCols cumulative W
  void *d_std_lnw = nullptr;          // and ln W(1) per row (context precision)
  int thin_groups = 0;
  qed_tuning tune{};
  unsigned *d_blk_start = nullptr;    // [4][nblk + 1] first record of each cell block
  unsigned *d_blk_cursor = nullptr;   // histogram / scatter cursors of the sort, one per key
  unsigned *d_phot_start = nullptr;   // [nblk + 2] photon sort starts (grid mode)
  int nb[3] = {0, 0, 0};
  int nblk = 0;
  int blk_keys = 1;                   // sort keys per cell block: its cells (grid mode), else 1
  int sorted = 0;                     // the stores are in cell-block order (up to the tail)
  void *d_clock = nullptr;            // {double t; long long step}: kernels advance it, so
                                      // captured CUDA graphs replay correctly
  size_t tables_bytes = 0;
  long long *d_tile = nullptr;        // compaction tile counts/offsets
  long long tile_cap = 0;
  int num_sms = 0;
  int blocks_photon = 0;              // grid sizes of the step kernels
  int blocks_massive = 0;
  int blocks_products = 0;
  int blocks_cells = 0;               // the cell-block pass: e-/e+, and ions alone
  int blocks_cells_ions = 0;
  int64_t step = 0;                   // host mirror of the clock (steps issued)
  int latched = 0;                    // a device error was observed
  int64_t steps_since_compact = 0;
  void *stage = nullptr;              // staging for pageable host I/O
  size_t stage_bytes = 0;
  cudaEvent_t ev_start = nullptr;     // recorded around the step kernels
  cudaEvent_t ev_photon = nullptr;
  cudaEvent_t ev_stop = nullptr;
  cudaEvent_t ev_stage[QED_NSTAGES] = {};   // qed_profile_stages: recorded at each stage
  std::vector<cudaEvent_t> ev_steps;  // qed_profile_stages with one block of events per step of a call
  cudaStream_t side = nullptr;        // the e-/e+/ion pass when it runs beside the photon pass
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int64_t launches = 0;               // kernels launched by this context
};

// A device status word folded into one qed_status (the most severe bit first).
inline int qed_fold_status(int bits) {
  if (bits & qed::kStCapacity) return QED_ERR_CAPACITY;
  if (bits & qed::kStNonfinite) return QED_ERR_NONFINITE;
  if (bits & qed::kStTimeout) return QED_ERR_TIMEOUT;
  if (bits & qed::kStPmGt1) return QED_ERR_PMGT1;
  if (bits & qed::kStCourant) return QED_ERR_COURANT;
  return QED_OK;
}

// Fold a status word read from the device and latch a failure in the
// context: qed_step refuses to run (QED_ERR_STATE) from then on.
inline int qed_latch_status(qed_ctx *c, int bits) {
  const int st = qed_fold_status(bits);
  if (st != QED_OK) c->latched = st;
  return st;
}

// Record the profiling event of one stage of the step, if the caller set one.
inline void qed_mark(qed_ctx *c, int stage, cudaStream_t s) {
  if (c->ev_stage[stage]) cudaEventRecord(c->ev_stage[stage], s);
}

// Internal launch interfaces (implemented in the .cu files).
int qed_build_tables(qed_ctx *c, cudaStream_t s);
int qed_launch_step(qed_ctx *c, const qed_fields *f, double dt, cudaStream_t s);
int qed_launch_yee(qed_ctx *c, const qed_fields *f, double dt, cudaStream_t s);
namespace qed {
int fold_grid_max(qed_ctx *c, cudaStream_t s);   // d_grid_max_next's stripes -> d_grid_max
}
int qed_launch_set(qed_ctx *c, int sp, const double *x, const double *p, const double *w,
                   const uint64_t *id, int64_t n, cudaStream_t s);
int qed_launch_get(qed_ctx *c, int sp, double *x, double *p, double *w, uint64_t *id, int64_t n,
                   cudaStream_t s);
int qed_launch_compact(qed_ctx *c, int sp, bool partition, cudaStream_t s);
int qed_launch_sort(qed_ctx *c, int sp, cudaStream_t s);
int qed_step_kernel_blocks(qed_ctx *c);
int qed_launch_chi_star(qed_ctx *c, cudaStream_t s);
int qed_launch_thin(qed_ctx *c, int sp, cudaStream_t s);
int qed_build_standard_tables(qed_ctx *c, cudaStream_t s);
int qed_launch_step_ext(qed_ctx *c, const qed_fields *f, double dt, cudaStream_t s);
int qed_step_kernel_blocks_ext(qed_ctx *c);
int qed_step_kernel_max_blocks_ext(qed_ctx *c, int *photon, int *massive);
int qed_step_kernel_max_blocks(qed_ctx *c, int *photon, int *massive);
