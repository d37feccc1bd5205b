/*
 * qed.h -- C ABI of the GB300 (sm_103a) QED Monte-Carlo particle step.
 *
 * The library implements the Monte-Carlo photon-emission and pair-production step of
 * Ridgers et al., "Modelling Gamma-Ray Photon Emission & Pair Production in High-Intensity
 * Laser-Matter Interactions" (arXiv:1311.5551), Sec. 3: per particle, field evaluation,
 * a relativistic Boris push, the quantum parameter eta (chi for photons), the optical-depth
 * advance with tabulated rates h(eta) and T(chi), and, where the optical depth is used up,
 * inverse-CDF sampling of the photon energy or the pair split, recoil, creation of the new
 * particles and a fresh optical depth.
 *
 * Conventions (all entry points):
 *  - Units: momenta in m_e c, photon momentum k = (h nu/m_e c^2) khat, fields E and cB in units
 *    of the Schwinger field E_s, time in hbar/(m_e c^2), length in hbar/(m_e c).
 *  - Every call is asynchronous on the caller's CUDA stream (passed as void*, NULL = legacy
 *    default stream) unless its comment says it synchronises.  Device memory comes from the
 *    caller's allocator (qed_allocator); the library never frees what it did not allocate.
 *  - Errors are returned as qed_status; qed_last_error() gives a message for the calling
 *    thread.  No C++ exception crosses this boundary.  Errors found on the device (capacity,
 *    non-finite values) are latched in a device flag and reported by the next call that
 *    synchronises (qed_check, qed_read_ledger, qed_species_download, qed_drain_new_particles).
 *  - Arrays are structure-of-arrays.  Particle positions and momenta have the species'
 *    precision (float for QED_MIXED, double for QED_FP64); optical depths are always double;
 *    ids are uint32.
 */
#ifndef QED_H
#define QED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QED_OK = 0,
  QED_ERR_INVALID_ARG = 1, /* a pointer, size or parameter is out of range */
  QED_ERR_OOM = 2,         /* the allocator returned NULL */
  QED_ERR_CAPACITY = 3,    /* new particles did not fit in a species' capacity */
  QED_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
  QED_ERR_CUDA = 5,        /* a CUDA runtime call failed (message in qed_last_error) */
  QED_ERR_NUMERIC = 6      /* a non-finite value was produced */
} qed_status;

typedef enum { QED_ELECTRON = 0, QED_POSITRON = 1, QED_PHOTON = 2 } qed_kind;

/* QED_MIXED: positions, momenta, push and rates in FP32, optical depth in FP64 and energy
 * sums compensated (the reduced-precision path); QED_FP64: everything in double. */
typedef enum { QED_FP64 = 0, QED_MIXED = 1 } qed_precision;

/* Device memory provider.  alloc(bytes, stream, user) returns device memory or NULL;
 * free(ptr, bytes, stream, user) releases it.  A NULL allocator uses cudaMallocAsync and
 * cudaFreeAsync on the given stream. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, size_t bytes, void* stream, void* user);
  void* user;
} qed_allocator;

/* ------------------------------------------------------------------------------------------
 * Look-up tables, Sec. 3 and Apps. A-B: h(eta), T(chi), the cumulative photon-energy
 * probability P_chi(eta, chi) and the pair-split probability P_f(f, chi).
 * eta nodes: n_eta log-spaced in [eta_min, eta_max].  For each eta node, n_xi nodes in
 * xi = 2 chi/eta, uniform in zeta = ln(xi/(1-xi)) from the cut-off xi_min(eta) (the ignored
 * photons carry energy_cut of the spectrum's energy, Sec. 3) to zeta = ln(90 eta).
 * chi nodes (T and P_f): n_chi log-spaced in [chi_min, chi_max]; P_f on n_f uniform f in
 * [0, 1/2] (p_f is symmetric about 1/2, App. B).
 * ------------------------------------------------------------------------------------------ */
typedef struct {
  int n_eta;          /* >= 2 */
  double eta_min, eta_max;
  int n_xi;           /* >= 2 */
  int n_chi;          /* >= 2 */
  double chi_min, chi_max;
  int n_f;            /* >= 2 */
  double energy_cut;  /* 1e-9 in the paper */
} qed_table_params;

/* Host image of a table set (double, row-major), used to export or import tables. */
typedef struct {
  double* ln_h;    /* [n_eta]          ln h(eta_i) */
  double* g;       /* [n_eta]          g(eta_i) (diagnostic) */
  double* zeta_lo; /* [n_eta]          logit of the cut-off xi_min(eta_i) */
  double* zeta_hi; /* [n_eta]          ln(90 eta_i) */
  double* P;       /* [n_eta * n_xi]   P_chi at the xi nodes (includes the ignored photons) */
  double* Q;       /* [n_eta * n_xi]   1 - P_chi, computed independently for precision */
  double* ln_T;    /* [n_chi]          ln T(chi_k) */
  double* Pf;      /* [n_chi * n_f]    P_f(f_j, chi_k) / P_f(1/2, chi_k) */
} qed_table_arrays;

typedef struct qed_tables qed_tables;

/* Build the tables on the host by Bessel-function quadrature (Apps. A-B) and upload FP64 and
 * FP32 images to the device.  Synchronises the stream.  *out is owned by the caller and
 * released with qed_tables_free. */
qed_status qed_tables_build(const qed_table_params* params, const qed_allocator* alloc, void* stream,
                            qed_tables** out);
/* Same, from caller-supplied table values (for instance published tables); arrays are read
 * during the call only.  Synchronises the stream. */
qed_status qed_tables_from_arrays(const qed_table_params* params, const qed_table_arrays* arrays,
                                  const qed_allocator* alloc, void* stream, qed_tables** out);
/* Copy the double host image into caller arrays sized per qed_table_arrays. */
qed_status qed_tables_export(const qed_tables* tables, qed_table_arrays* dst);
void qed_tables_free(qed_tables* tables);

/* ------------------------------------------------------------------------------------------
 * Particle species: SoA arrays of capacity `capacity` in device memory plus an append region
 * of `append_capacity` slots that holds the particles created for this species during one
 * step (Sec. 3.2: macro-photons and macro-pairs created by the emission step).
 * ------------------------------------------------------------------------------------------ */
typedef struct qed_species qed_species;

typedef struct {
  void* x; void* y; void* z;     /* positions (species precision) */
  void* ux; void* uy; void* uz;  /* momenta u = p/(m c), or k for photons (species precision) */
  double* tau;                   /* remaining optical depth; +inf marks a converted photon */
  uint32_t* id;                  /* particle id (Philox stream key) */
} qed_soa;

/* Device view of a species' arrays (the arrays stay owned by the species).  Inside the library
 * a QED_MIXED species keeps tau as a compensated pair of floats (hi, lo) in the same 8 bytes;
 * upload and download convert from and to double, the view exposes the stored form. */
typedef struct {
  qed_soa arrays;
  size_t capacity;
  int kind, precision;
} qed_species_view;

qed_status qed_species_alloc(qed_kind kind, qed_precision precision, size_t capacity, size_t append_capacity,
                             const qed_allocator* alloc, void* stream, qed_species** out);
void qed_species_free(qed_species* sp);
/* Replace the contents with n particles from src (host or device pointers of the species'
 * precision; src.tau and src.id may be NULL: tau is then set to 0 and ids to 0..n-1).
 * Sets next_id to max(id)+1 (n when ids are generated).  The host arrays are read before the
 * call returns only if they are pageable; pinned or device sources are copied asynchronously
 * and must stay valid until the stream reaches the copy. */
qed_status qed_species_upload(qed_species* sp, const qed_soa* src, size_t n, uint32_t next_id, void* stream);
/* Copy up to cap live particles into dst (host or device); writes the count to *n_out.
 * Synchronises the stream. */
qed_status qed_species_download(qed_species* sp, const qed_soa* dst, size_t cap, size_t* n_out, void* stream);
/* Number of particles held (converted photons are counted until compaction).  Synchronises. */
qed_status qed_species_count(const qed_species* sp, size_t* n_out, void* stream);
qed_status qed_species_view_get(const qed_species* sp, qed_species_view* view);
/* Checkpoint and resume (bit-exact): the held particles in their stored form, laid out as a
 * 64-byte header (kind, precision, n, next_id, n_dead) followed by x, y, z, ux, uy, uz (species
 * precision), tau (8 bytes, stored form) and id arrays of n entries each.  qed_species_save
 * writes at most cap_bytes to dst (host or device) and the size used to *bytes_out (pass
 * dst = NULL to query the size); it synchronises.  qed_species_restore reads such a checkpoint
 * into a species of the same kind and precision (the source must stay valid until the stream
 * reaches the copies).  Because the Philox streams are keyed by (seed, id, step), a run resumed
 * from a checkpoint is bit-identical to an uninterrupted run. */
qed_status qed_species_save(qed_species* sp, void* dst, size_t cap_bytes, size_t* bytes_out, void* stream);
qed_status qed_species_restore(qed_species* sp, const void* src, size_t bytes, void* stream);
/* Initial optical depths, Sec. 3: tau = -ln U with U from the Philox stream
 * (key = (seed, scenario), counter = (id, 0, kind, 1)). */
qed_status qed_species_init_tau(qed_species* sp, uint64_t seed, uint64_t scenario, void* stream);
/* Stable removal of converted photons (tau = +inf).  Uses the species' scratch arrays. */
qed_status qed_species_compact(qed_species* sp, void* stream);

/* Macroparticle weights (the physical particles a macroparticle stands for).  Uploads set
 * every weight to 1; children (emitted photons, pairs) inherit their parent's weight.  Arrays
 * in the species precision, host or device.  A species holds weight arrays (4 or 8 bytes per
 * particle and append slot, from its allocator) only from the first call that sets, merges or
 * restores weights other than 1, or from the first step with a partner species that holds
 * them; until then every weight is 1 and takes no memory. */
qed_status qed_species_set_weights(qed_species* sp, const void* w, size_t n, void* stream);
qed_status qed_species_get_weights(qed_species* sp, void* dst, size_t cap, size_t* n_out, void* stream);
/* Physical totals of the held particles (converted photons excluded): out[0] = sum w,
 * out[1] = sum w * energy (gamma for e+-, |k| for photons), out[2..4] = sum w * momentum.
 * FP64, fixed summation order.  Synchronises. */
qed_status qed_species_totals(qed_species* sp, double out[5], void* stream);

/* Macroparticle merging (any species; stated here for photons, electrons and positrons use
 * their energy gamma and the two members sit on the mass shell).  Sec. 3.1 names merging
 * macroparticles as the way to keep a growing
 * population (an e+e- cascade) bounded, and does not implement it; this is one definition that
 * conserves what the ledger tracks.  Photons are grouped by a cell of a position grid
 * (floor((x - origin)/cell) per axis; photons outside are not merged), a direction bin (the face
 * of the cube [-1,1]^3 that k points through and an n_face x n_face bin of the other two
 * components divided by the largest) and an energy bin (the binary exponent of |k| and one of
 * n_sub sub-bins of its mantissa); these use exact operations only, so any IEEE double
 * implementation finds the same groups.  Every group of at least min_group (>= 3) photons
 * becomes two photons of half its weight at its weighted mean position that carry exactly its
 * total weight W, momentum P and energy E: energy E/W each, momenta P/W + d and P/W - d with d
 * perpendicular to P.  They are the group's two lowest-index photons (keeping ids and optical
 * depths); the others are removed and the remaining photons keep their order.  *groups_out:
 * groups merged.  Takes temporary device memory of 12 bytes per photon from the allocator the
 * species was created with (released before the call returns); synchronises. */
typedef struct {
  double origin[3], cell[3];
  int32_t n_cells[3];
  int32_t n_face;
  int32_t n_sub;
  int32_t min_group;
} qed_merge_params;
qed_status qed_species_merge(qed_species* sp, const qed_merge_params* params, uint64_t* groups_out, void* stream);

/* ------------------------------------------------------------------------------------------
 * Fields: the analytic stand-ins for the PIC field gather (Sec. 3.2).
 *  QED_FIELD_UNIFORM   : E and cB constant.
 *  QED_FIELD_ROTATING_E: E = E0 (cos(omega t + phase0), sin(omega t + phase0), 0), B = 0.
 *  QED_FIELD_PLANE_LP  : wave along +x, phase phi = omega (t - x) - phi_start,
 *                        E_y = cB_z = E0 env(phi) cos(phi).
 *  QED_FIELD_PLANE_CP  : E = E0 env (0, cos phi, sin phi), cB = E0 env (0, -sin phi, cos phi).
 *  env(phi) = sin^2(pi phi/phi_len) on 0 < phi < phi_len and 0 outside; phi_len <= 0: env = 1.
 *  QED_FIELD_GRID      : the PIC field gather of Sec. 3.2 (each particle takes the fields
 *                        interpolated from the grid to its position).  `grid` is a device array
 *                        of six components Ex, Ey, Ez, cBx, cBy, cBz, each n[0]*n[1]*n[2] values
 *                        (x fastest) in the species precision (float for QED_MIXED, double for
 *                        QED_FP64), owned by the caller and read during the step.  Yee
 *                        staggering: E_c sits at node + spacing/2 along axis c, cB_c at node +
 *                        spacing/2 along the two other axes; node (i, j, k) is at
 *                        origin + (i, j, k) * spacing in window coordinates (the stored
 *                        positions).  shape = 1: cloud-in-cell (linear weights over 2 nodes per
 *                        axis); shape = 2: triangular-shaped cloud (quadratic weights over the
 *                        nearest node and its two neighbours).  Stencil nodes outside the grid
 *                        contribute nothing, so fields fall to zero outside it.  The fields do
 *                        not depend on t: the caller updates the grid between steps.
 * ------------------------------------------------------------------------------------------ */
typedef enum {
  QED_FIELD_UNIFORM = 0, QED_FIELD_ROTATING_E = 1, QED_FIELD_PLANE_LP = 2, QED_FIELD_PLANE_CP = 3,
  QED_FIELD_GRID = 4
} qed_field_kind;

typedef struct {
  int kind;
  double E[3], B[3];
  double E0, omega, phase0, phi_start, phi_len;
  /* QED_FIELD_GRID only */
  const void* grid;
  int32_t n[3];
  int32_t shape;
  double origin[3], spacing[3];
} qed_field_desc;

/* One step n: t_n = t0 + n dt.  Positions are stored relative to a moving window
 * x_w(t) = window_x0 + window_v t along x (use 0, 0 for absolute positions); keeping them
 * small keeps FP32 positions and the FP32 plane-wave phase accurate. */
typedef struct {
  double dt, t0;
  uint64_t step;       /* n; its Philox counter word */
  uint64_t seed;       /* Philox key word 0 */
  uint64_t scenario;   /* Philox key word 1 */
  qed_field_desc field;
  int emit_photons;    /* photon emission by e+- (Sec. 3) */
  int make_pairs;      /* pair creation by photons (Sec. 3) */
  int drain_photons;   /* new photons go to the drain species instead of being pushed (Sec. 3.1) */
  int recoil_energy;   /* 0: recoil p_f = p_i - (h nu/c) phat_i (Sec. 3); 1: energy-conserving */
  double window_x0, window_v;
} qed_step_params;

/* Per-step ledger (FP64 sums over the step just taken). */
typedef struct {
  double n[3];            /* live e-, e+, photons after the step */
  double energy[3];       /* their energy: sum gamma (e+-) or sum eps (photons) */
  double emitted_n, emitted_energy; /* photons created (kept or drained) */
  double dropped_n;       /* emission events below the table cut-off (photon ignored, Sec. 3) */
  double emit_defect;     /* sum (gamma_f + eps) - gamma_i over emissions (Sec. 3.1) */
  double pairs_n, pair_energy, pair_defect;
  double drained_n, drained_energy;
  double oor_eta, oor_chi; /* look-ups beyond the top of the tables (clamped) */
} qed_ledger;

/* One Monte-Carlo step of electrons sp[0], positrons sp[1] and photons sp[2] (Sec. 3): field
 * evaluation, Boris push (photons move at c along k), eta/chi, tau -= lambda dt with
 * lambda_gamma = (sqrt3 alpha/2pi)(eta/gamma) h(eta) and lambda_pm = alpha (chi/eps) T(chi)
 * (eqs. rate_photons and pair_prod_rate), at most one event per particle per step, sampling,
 * recoil and creation of the new particles, which join at the next step ordered by
 * (parent species, parent index) with consecutive ids.  sp[3] receives the new photons when
 * drain_photons is set (it may be NULL otherwise).  Species must share one precision. */
qed_status qed_step(const qed_tables* tables, qed_species* const* sp, const qed_step_params* params, void* stream);
/* n_steps consecutive steps starting at params->step. */
qed_status qed_run(const qed_tables* tables, qed_species* const* sp, const qed_step_params* params,
                   uint64_t n_steps, void* stream);
/* Ledger of the last step taken on these species.  Synchronises the stream. */
qed_status qed_read_ledger(qed_species* const* sp, qed_ledger* out, void* stream);
/* Move the particles held by a drain species into dst (host or device, capacity cap) and
 * empty it; *n_out receives the number moved.  Synchronises the stream. */
qed_status qed_drain_new_particles(qed_species* drained, const qed_soa* dst, size_t cap, size_t* n_out,
                                   void* stream);
/* Synchronise and report (and clear) errors latched on the device by earlier calls on sp. */
qed_status qed_check(qed_species* const* sp, int n_species, void* stream);

/* ------------------------------------------------------------------------------------------
 * Batches: many independent scenarios (for example a parameter scan of collisions, or the
 * requests of a serving loop), each with its own species, field and steps, advanced together.
 * Each batch step is five launches for all scenarios: a tile schedule that lays the live
 * scenarios' 256-particle tiles end to end in one tile space, the step (a persistent grid that
 * strides through that space, so every block gets an equal share in one wave), and the three
 * merge kernels (per-scenario plan, event-mask prefixes and the ordered scatter, each striding
 * through all scenarios together); qed_batch_run replays them from a captured CUDA graph.  A
 * scenario gives the same particles alone or in any mix, and, with the default grid, the same
 * ledger bit for bit as qed_run (block p of the grid takes the same tiles of the scenario either
 * way).
 * ------------------------------------------------------------------------------------------ */
typedef struct qed_batch qed_batch;
qed_status qed_batch_create(const qed_tables* tables, qed_precision precision, int slots,
                            const qed_allocator* alloc, void* stream, qed_batch** out);
/* Put a scenario in a slot: species sp[0..2] (e-, e+, photons) and sp[3] (photon drain or NULL)
 * stay owned by the caller and must outlive the slot; its first step is params->step and it
 * advances n_steps steps (Sec. 3 per step, as qed_step).  Re-attach after compacting, merging or
 * setting the weights of a species (its arrays may move). */
qed_status qed_batch_attach(qed_batch* b, int slot, qed_species* const* sp, const qed_step_params* params,
                            uint64_t n_steps, void* stream);
qed_status qed_batch_detach(qed_batch* b, int slot, void* stream);
/* n_steps batch steps; a slot whose remaining steps reach 0 stops. */
qed_status qed_batch_run(qed_batch* b, uint64_t n_steps, void* stream);
/* Remaining steps per slot (slots entries).  Synchronises. */
qed_status qed_batch_remaining(qed_batch* b, uint32_t* out, void* stream);
/* Launch configuration: the step kernel's grid (blocks striding through the batch step's tiles,
 * at most one ledger partial each; 0: the default, one wave at full occupancy, which is the
 * single-scenario step's grid, so a slot's ledger equals its qed_run ledger bit for bit) and
 * batch steps per captured graph (0: no graph). */
qed_status qed_batch_config(qed_batch* b, int target_blocks, int graph_steps);
/* Multi-step passes in every batch step (chunk 0: off; 2..64): each live slot first takes its
 * event-free stretch of up to chunk steps in one pass (as qed_run_multistep, decided on the device
 * per slot, no host synchronisation), then the regular step, so one batch step advances a slot by
 * one to chunk + 1 steps; particles are identical to qed_run's.  Run batch steps until
 * qed_batch_remaining reports zero. */
qed_status qed_batch_multistep(qed_batch* b, int chunk);
/* Autotuner: times candidate (blocks, graph steps) on the live batch, trial_steps real batch
 * steps each, and keeps the fastest; the chosen values are returned.  Synchronises. */
qed_status qed_batch_tune(qed_batch* b, int trial_steps, int* target_blocks, int* graph_steps, void* stream);
void qed_batch_free(qed_batch* b);

/* Multi-step run: the same n_steps steps as qed_run, with identical particle results, but every
 * stretch of steps in which no particle has an event is taken in one pass over the particles
 * (positions, momenta and optical depths stay in registers for up to `chunk` steps, 2 <= chunk
 * <= 64).  The paper's step (Sec. 3) creates children only at events, and a step without events
 * is a push, an eta/chi evaluation and an optical-depth decrement per particle, independent of
 * every other particle; only steps with events need the ordered merge.  Each stretch is found by
 * a read-only probe pass (the first step at which any particle would have an event), then
 * committed; a step with events runs on the per-step kernels.  The call synchronises the stream
 * once per probe.  After it, qed_read_ledger reports the last step (push counts of a committed
 * stretch cover all of its steps).  Work done by the multi-step passes is reported separately
 * by qed_work_read_split. */
qed_status qed_run_multistep(const qed_tables* tables, qed_species* const* sp, const qed_step_params* params,
                             uint64_t n_steps, int chunk, void* stream);

/* ------------------------------------------------------------------------------------------
 * Allocation-free emission step.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory -- a host simulation that has already claimed the
 * device memory for its own pool, or a time loop that must keep its memory footprint fixed and
 * cannot pay for cudaMalloc's implicit device-wide synchronisation.
 *
 * One step of photon emission (no pair creation) for n_electrons <= 65536 electrons held in the
 * caller's device arrays (16-byte aligned, species precision; tau in the stored form: double for
 * QED_FP64, a (hi, lo) float pair for QED_MIXED, see qed_species_view), updated in place.  The
 * new photons are appended in parent order to the caller's photon arrays from index
 * photon_counter[0]; photon_counter is a device array of 3 uint32: [count, next id, error bits]
 * (QED_ERR_* as 1 << code), updated on the stream.  Nothing is allocated: all scratch lives in
 * one fixed array of about 4.3 MB inside the library, which every GPU that loads the library
 * holds until the process exits.  The first call on a device looks up that array's address
 * (cudaGetSymbolAddress); make the first call on each device before any stream capture.  All
 * calls share the array and it keeps the last call's contents (each call clears what must start
 * at zero), so calls that overlap on the GPU (unordered streams) race.  Returns
 * QED_ERR_INVALID_ARG for more than 65536 electrons or misaligned arrays.
 * ------------------------------------------------------------------------------------------ */
qed_status qed_step_emit_noalloc(const qed_tables* tables, qed_precision precision, const qed_soa* electrons,
                                 size_t n_electrons, const qed_soa* photons, size_t photon_capacity,
                                 uint32_t* photon_counter, const qed_step_params* params, void* stream);

/* ------------------------------------------------------------------------------------------
 * Diagnostics that run the same device functions as the step (used by parity tests).
 * All pointers are device pointers to double arrays of length n.
 * ------------------------------------------------------------------------------------------ */
/* Per particle at time t: fields E, cB (3n each, interleaved xyz), eta (e+-) or chi (photons),
 * gamma or eps, and the rate lambda_gamma or lambda_pm, in the given precision. */
qed_status qed_eval_particles(const qed_tables* tables, qed_precision precision, qed_kind kind,
                              const qed_field_desc* field, double t, double window_x0, double window_v,
                              size_t n, const double* x, const double* y, const double* z, const double* ux,
                              const double* uy, const double* uz, double* out_E, double* out_B,
                              double* out_param, double* out_energy, double* out_rate, void* stream);
/* Inverse-CDF samples: which = 0: xi = 2chi/eta for (eta[i], U[i]) (out_ok[i] = 0 below the
 * cut-off); which = 1: pair split f for (chi[i], U[i]).  Rate look-ups (Sec. 3, "linearly
 * interpolating" the tabulated h and T): which = 2: h(eta[i]); which = 3: T(chi[i]); U is not
 * read (may be NULL) and out_ok[i] is the look-up's range flag (-1 below, 1 above the table,
 * 0 inside). */
qed_status qed_sample(const qed_tables* tables, qed_precision precision, int which, size_t n, const double* param,
                      const double* U, double* out, int32_t* out_ok, void* stream);
/* Philox4x64-10 blocks for counters ctr[4i..4i+3] under key[0..1] (host array); device in/out. */
qed_status qed_philox(size_t n, const uint64_t* ctr, const uint64_t key[2], uint64_t* out, void* stream);

/* Work done by steps whose sp[0] is `electrons`, cumulative since the last reset: out[0] e+-
 * pushes, out[1] photon pushes (converted photons excluded), out[2] particles created.
 * Synchronises. */
qed_status qed_work_read(qed_species* electrons, uint64_t out[3], int reset, void* stream);
/* As qed_work_read, plus out[3] e+- pushes and out[4] photon pushes made by multi-step passes
 * (already counted in out[0] and out[1]), and out[5] photon pushes of the per-step kernel in a
 * field, whose optical depth changed and was written back (a photon outside every field keeps
 * its optical depth, and the step stores only its position). */
qed_status qed_work_read_split(qed_species* electrons, uint64_t out[6], int reset, void* stream);
/* Step-kernel timing: while enabled, every step-kernel launch is bracketed by CUDA events on its
 * stream.  qed_timing_read waits for the recorded events and returns the summed kernel time (ms)
 * and the number of launches timed since the last reset. */
qed_status qed_timing_enable(int on);
qed_status qed_timing_read(double* step_kernel_ms, uint64_t* launches, int reset);
/* The same for the multi-step passes of qed_run_multistep (probe and commit launches). */
qed_status qed_timing_read_multistep(double* ms, uint64_t* passes, int reset);

/* Failure-detection self-test: runs the bounded mbarrier wait that every pipeline wait of the
 * step uses on a barrier that completes and on one that nothing ever arrives at, with `polls`
 * polls.  *bits_out: 1 = the completed wait succeeded, 2 = the unsatisfiable wait gave up
 * (3 = both, as it should).  The kernel returns either way; the context stays usable. */
qed_status qed_selftest_wait(uint32_t polls, uint32_t* bits_out, void* stream);

/* Kernel launches issued by this library since it was loaded (for launch accounting). */
uint64_t qed_launch_count(void);
const char* qed_version(void);
const char* qed_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QED_H */
