// qed_internal.h -- structures shared by the library's translation units (not part of the ABI).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "qed.h"

// The host-only translation units do not include the CUDA runtime headers; this is the same
// declaration the runtime makes.
struct CUstream_st;
typedef struct CUstream_st* cudaStream_t;

namespace qedlib {

// ------------------------------------------------------------------ host table image
struct TableHost {
  qed_table_params p{};
  std::vector<double> ln_h, g, zeta_lo, zeta_hi, P, Q, ln_T, Pf;
  void resize(const qed_table_params& prm);
};
bool validate_table_params(const qed_table_params& p, std::string& err);
bool build_tables_host(const qed_table_params& p, TableHost& out, std::string& err);

// ------------------------------------------------------------------ device structures
// Look-up tables in precision R (device pointers + grid scalars).
template <typename R>
struct TabDev {
  const R* ln_h;     // [n_eta]
  const R* ln_T;     // [n_chi]
  const R* P;        // [n_eta * n_xi]
  const R* Q;        // [n_eta * n_xi]
  const R* zeta_lo;  // [n_eta]
  const R* zeta_hi;  // [n_eta]
  const R* Pf;       // [n_chi * n_f]
  int n_eta, n_xi, n_chi, n_f;
  R ln_eta_min, inv_d_eta, eta_min;
  R ln_chi_min, inv_d_chi, chi_min, chi_max, T_at_chi_max;
};

// Per-species counters in device memory.
struct DevCounters {
  uint32_t n;        // particles held, including converted photons awaiting compaction
  uint32_t next_id;  // id given to the next particle created
  uint32_t n_app;    // particles appended to this species' append region during the step
  uint32_t n_dead;   // converted photons held
  uint32_t err;      // latched error bits (QED_ERR_* as 1u << code)
  uint32_t pad[3];
};

constexpr int kRangeShift = 8;  // one range = 256 warp chunks = 8192 parents
constexpr int kLedgerN = 18;

// Species arrays in precision R plus the scratch used by one step.
template <typename R>
struct SpeciesDev {
  R *x, *y, *z, *ux, *uy, *uz;
  double* tau;
  uint32_t* id;
  uint32_t cap;
  DevCounters* cnt;
  // as a parent: which lanes of each 32-particle chunk created children this step
  uint32_t* evmask;   // [cap/32 + 1]
  uint32_t* rangesum; // [ranges]  children per range of 256 chunks (integer atomics)
  uint32_t* rprefix;  // [ranges]  exclusive prefix of rangesum
  uint32_t* wprefix;  // [cap/32 + 1] exclusive prefix of popc(evmask)
  // as a destination: particles created for this species during the step
  R *ax, *ay, *az, *aux, *auy, *auz;
  double* atau;
  uint32_t* aparent;  // parent index | (parent is a positron) << 31
  uint32_t acap;
  // macroparticle weights (NULL: every particle has weight 1); children inherit their parent's
  R* w;   // [cap]
  R* aw;  // [acap]
};

// Finalisation plan written by the first finalisation kernel.
struct FinalizePlan {
  uint32_t n_old[3];        // destination counts before the merge (e-, e+, photon destination)
  uint32_t next_id_old[3];
  uint32_t m[3];            // particles merged into each destination
  uint32_t from_electrons;  // photon children whose parents are electrons (ranked first)
  uint32_t ranges[3];       // ranges per parent species
  uint32_t events[3];       // events of each parent species this step
  uint32_t pad;
};

// Analytic field parameters (Sec. 3.2 stand-in for the PIC gather).
struct FieldDev {
  int kind;
  double E[3], B[3];
  double E0, omega, phase0, phi_start, phi_len;
  // QED_FIELD_GRID: six Yee-staggered components (species precision), nodes, shape, geometry
  const void* grid;
  int n[3];
  int shape;
  double origin[3], spacing[3];
};

// Host: descriptor -> device form, and its validation (shared by every entry point that steps).
FieldDev field_dev(const qed_field_desc& f);
qed_status check_field(const qed_field_desc& f, const char* who);

template <typename R>
struct StepArgs {
  SpeciesDev<R> sp[4];  // e-, e+, photons, drain (photon destination when draining)
  TabDev<R> tab;
  FieldDev field;
  double dt, t0, win_x0, win_v;
  R dt_r, win_v_r;  // dt and the window velocity in the working precision (set on the host)
  uint64_t seed, scenario, step;
  int emit, pairs, drain, recoil_energy;
  double* ledger_part;  // [gridDim.x * kLedgerN]
  double* ledger;       // [kLedgerN]
  FinalizePlan* plan;
  unsigned long long* work;  // [5] cumulative e+- pushes, photon pushes, particles created, and the
                             // e+- and photon pushes made by multi-step passes (part of [0], [1])
  int multi;                 // this finalisation follows a multi-step commit
};

// What one batch step does with a slot, written by the tile schedule at the start of the step:
// the slot's 256-particle tiles occupy [tile_base, tile_base + T[0] + T[1] + T[2]) of the batch
// step's tile space (species in order e-, e+, photons), its event-mask ranges
// [range_base, range_base + Rg[0] + Rg[1] + Rg[2]) of the range space; n are the particles
// held (the step's parents).
struct SlotPlan {
  uint32_t live;
  uint32_t tile_base;
  uint32_t T[3];
  uint32_t n[3];
  uint32_t range_base;
  uint32_t Rg[3];
};
constexpr int kBatchTotals = 4;  // [tiles, ranges, children (after the plan), spare]

// Many independent scenarios ("slots") stepped together: per-slot arguments live in device
// memory.  The per-step path puts the tiles of all live slots in one tile space that a
// persistent grid strides through; the multi-step passes give every live slot a share of the
// blocks proportional to its tiles.
template <typename R>
struct BatchCtl {
  StepArgs<R>* args;     // [S] per-slot arguments (their step field is the next step to take)
  uint32_t* remaining;   // [S] steps left per slot (0: idle)
  uint32_t* live;        // [S] slot takes part in the current batch step (set by the schedule)
  uint32_t* blocks;      // [S+1] exclusive prefix of the step-kernel blocks per slot (multi-step)
  SlotPlan* splan;       // [S] tile and range layout of the current batch step
  void* scal;            // [S] per-slot field scalars of the current step (StepScalars<R>)
  uint32_t* tot;         // [kBatchTotals] sizes of the current batch step's spaces
  TabDev<R> tab;         // the batch's tables (shared by every slot)
  int S;                 // slots
  int target_blocks;     // step-kernel grid (blocks striding through the tile space)
  int max_parts;         // ledger partials available per slot
  int grid_fields;       // some slot gathers its fields from a grid (selects that instantiation)
  uint32_t* first_event; // [S] multi-step probe result per slot
  uint32_t* tried;       // [S] stretch the slot's probe tried this batch step (0: not probed)
  uint32_t* skip;        // [S] batch steps the slot waits before probing again
  uint32_t* span;        // [S] stretch the slot's next probe tries (adapts to what probes find)
  int fuse_k;            // multi-step stretch per batch step (0: per-step only)
};

template <typename R>
void launch_step(const StepArgs<R>& a, int grid, int block, size_t smem, cudaStream_t s);
template <typename R>
void launch_batch_step(const BatchCtl<R>& c, int n_eta, int n_chi, cudaStream_t s);
size_t step_scalars_bytes(int precision);
template <typename R>
void launch_finalize(const StepArgs<R>& a, int step_grid, cudaStream_t s);
// Multi-step pass over K <= fuse_max_steps() steps: the probe (commit = false) sets
// *first_event to the first step with an event (K if none); the commit advances K event-free
// steps and writes the ledger partials of the last.  Returns the grid (ledger partials) used.
template <typename R>
int launch_fused(const StepArgs<R>& a, int K, bool commit, uint32_t* first_event, int max_parts, cudaStream_t s);
int fuse_max_steps();
void launch_selftest_wait(uint32_t polls, uint32_t* bits, cudaStream_t s);
template <typename R>
void launch_init_tau(const SpeciesDev<R>& sp, int kind, uint64_t seed, uint64_t scenario, cudaStream_t s);
template <typename R>
void launch_eval(const TabDev<R>& tab, const FieldDev& f, int kind, double t, double wx0, double wv, size_t n,
                 const double* x, const double* y, const double* z, const double* ux, const double* uy,
                 const double* uz, double* oE, double* oB, double* oparam, double* oenergy, double* orate,
                 cudaStream_t s);
template <typename R>
void launch_sample(const TabDev<R>& tab, int which, size_t n, const double* param, const double* U, double* out,
                   int32_t* ok, cudaStream_t s);
void launch_philox(size_t n, const uint64_t* ctr, uint64_t k0, uint64_t k1, uint64_t* out, cudaStream_t s);
template <typename R>
void launch_compact(const SpeciesDev<R>& sp, const SpeciesDev<R>& out, uint32_t* seg_count, uint32_t* seg_prefix,
                    cudaStream_t s);

void launch_tau_convert(int precision, double* tau, size_t n, bool to_double, cudaStream_t s);

// Macroparticle weights: fill, physical totals, photon merging (see qed_species_merge).
template <typename R>
void launch_fill(R* p, size_t n, R v, cudaStream_t s);
template <typename R>
void launch_totals(const SpeciesDev<R>& sp, int massless, double* partials, int blocks, cudaStream_t s);
struct MergeDev {
  double origin[3], cell[3];
  int n_cells[3], n_face, n_sub, min_group;
};
template <typename R>
void launch_merge(const SpeciesDev<R>& sp, const MergeDev& m, uint64_t* keys, uint32_t* idx, uint32_t N,
                  int massless, unsigned long long* groups, cudaStream_t s);

// Device images of a table set (defined with qed_tables in qed_api.cu).
struct TablesDev {
  TabDev<double> d64;
  TabDev<float> d32;
  template <typename R> const TabDev<R>& get() const;
};
template <> inline const TabDev<double>& TablesDev::get<double>() const { return d64; }
template <> inline const TabDev<float>& TablesDev::get<float>() const { return d32; }
TablesDev tables_dev(const qed_tables* t);
// Records the calling thread's error message (qed_last_error) and returns st.
qed_status set_error(qed_status st, const std::string& msg);
int step_grid_size(int precision);
void count_launch(int n = 1);

}  // namespace qedlib
