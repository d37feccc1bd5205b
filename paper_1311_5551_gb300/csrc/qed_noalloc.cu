// qed_noalloc.cu -- an allocation-free variant of the emission step for callers that must not
// allocate device memory.
//
// The regular entry points keep their per-step scratch (event masks, prefix sums, the append
// region of new photons, ledger partials, the merge plan, counters) inside species objects that
// are allocated through a qed_allocator.  Some host codes cannot grant that: a simulation that has
// reserved the whole device memory for its own pool, or a time loop that must not change its
// memory footprint or pay for cudaMalloc's implicit device synchronisation.  For them
// qed_step_emit_noalloc runs the same kernels with all scratch in the fixed-size array below,
// which is part of the loaded library image (every GPU that loads the library holds it, about
// 4.3 MB, until the process exits).
#include <cuda_runtime.h>

#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "qed_internal.h"

using namespace qedlib;

namespace {

constexpr size_t kMaxElectrons = 65536;  // per call
constexpr size_t kWords = kMaxElectrons / 32 + 2;
constexpr size_t kRanges = (kWords >> kRangeShift) + 2;
constexpr size_t kMaxGrid = 2048;        // step-kernel blocks (ledger partials)
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
// layout of the scratch array (byte offsets)
constexpr size_t kOffCounters = 0;                                           // 4 DevCounters
constexpr size_t kOffMasks = align256(kOffCounters + 4 * sizeof(DevCounters));  // evmask, wprefix
constexpr size_t kOffRanges = align256(kOffMasks + 2 * kWords * 4);          // rangesum, rprefix
constexpr size_t kOffAppend = align256(kOffRanges + 2 * kRanges * 4);        // photon append region
constexpr size_t kAppendBytes = kMaxElectrons * (6 * 8 + 8 + 4) + 8 * 256;   // sized for FP64
constexpr size_t kOffLedger = align256(kOffAppend + kAppendBytes);           // partials + ledger
constexpr size_t kLedgerBytes = (kMaxGrid + 1) * kLedgerN * 8;
constexpr size_t kOffPlan = align256(kOffLedger + kLedgerBytes);
constexpr size_t kOffWork = align256(kOffPlan + sizeof(FinalizePlan));
constexpr size_t kOffEmpty = align256(kOffWork + 5 * 8);                     // masks of the empty species
constexpr size_t kScratchBytes = align256(kOffEmpty + 64);

// The scratch.  Host code must not pass this name to a kernel: on the host it is only a
// stand-in for the device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[128] = {};  // device address of the scratch, per device ordinal

__global__ void noalloc_begin_kernel(DevCounters* c, uint32_t n_e, const uint32_t* photon_counter) {
  // electrons, positrons (empty), photons (empty, receives the append), drain = caller's arrays
  for (int k = 0; k < 4; ++k) { c[k].n = 0; c[k].next_id = 0; c[k].n_app = 0; c[k].n_dead = 0; c[k].err = 0; }
  c[0].n = n_e;
  c[3].n = photon_counter[0];
  c[3].next_id = photon_counter[1];
}

__global__ void noalloc_end_kernel(const DevCounters* c, uint32_t* photon_counter) {
  photon_counter[0] = c[3].n;
  photon_counter[1] = c[3].next_id;
  uint32_t err = 0;
  for (int k = 0; k < 4; ++k) err |= c[k].err;
  photon_counter[2] |= err;
}

template <typename R>
void bind_species(SpeciesDev<R>& s, DevCounters* cnt, uint32_t* masks, uint32_t* ranges, size_t words,
                  size_t nranges) {
  s.cnt = cnt;
  s.evmask = masks;
  s.wprefix = masks + words;
  s.rangesum = ranges;
  s.rprefix = ranges + nranges;
}

template <typename R>
qed_status run_noalloc(const TablesDev& tv, const qed_soa* e, size_t n, const qed_soa* ph, size_t ph_cap,
                       uint32_t* counter, const qed_step_params* p, unsigned char* base, cudaStream_t s) {
  DevCounters* cnt = reinterpret_cast<DevCounters*>(base + kOffCounters);
  uint32_t* masks = reinterpret_cast<uint32_t*>(base + kOffMasks);
  uint32_t* ranges = reinterpret_cast<uint32_t*>(base + kOffRanges);
  uint32_t* empty = reinterpret_cast<uint32_t*>(base + kOffEmpty);
  StepArgs<R> a{};
  // electrons: the caller's arrays, updated in place
  SpeciesDev<R>& el = a.sp[0];
  el.x = (R*)e->x; el.y = (R*)e->y; el.z = (R*)e->z; el.ux = (R*)e->ux; el.uy = (R*)e->uy; el.uz = (R*)e->uz;
  el.tau = e->tau; el.id = e->id; el.cap = (uint32_t)n; el.acap = 0;
  bind_species(el, cnt + 0, masks, ranges, kWords, kRanges);
  // positrons: empty (no pairs in this variant)
  bind_species(a.sp[1], cnt + 1, empty, empty + 4, 2, 2);
  // photons: empty, but their append region (in the scratch) collects the new photons
  SpeciesDev<R>& pg = a.sp[2];
  bind_species(pg, cnt + 2, empty, empty + 4, 2, 2);
  unsigned char* ap = base + kOffAppend;
  auto take = [&](size_t bytes) { unsigned char* q = ap; ap += align256(bytes); return q; };
  pg.ax = (R*)take(kMaxElectrons * sizeof(R)); pg.ay = (R*)take(kMaxElectrons * sizeof(R));
  pg.az = (R*)take(kMaxElectrons * sizeof(R)); pg.aux = (R*)take(kMaxElectrons * sizeof(R));
  pg.auy = (R*)take(kMaxElectrons * sizeof(R)); pg.auz = (R*)take(kMaxElectrons * sizeof(R));
  pg.atau = (double*)take(kMaxElectrons * 8); pg.aparent = (uint32_t*)take(kMaxElectrons * 4);
  pg.acap = (uint32_t)kMaxElectrons;
  // drain: the caller's photon arrays
  SpeciesDev<R>& dr = a.sp[3];
  dr.x = (R*)ph->x; dr.y = (R*)ph->y; dr.z = (R*)ph->z; dr.ux = (R*)ph->ux; dr.uy = (R*)ph->uy; dr.uz = (R*)ph->uz;
  dr.tau = ph->tau; dr.id = ph->id; dr.cap = (uint32_t)ph_cap; dr.cnt = cnt + 3;
  a.tab = tv.get<R>();
  a.field = field_dev(p->field);
  a.dt = p->dt; a.t0 = p->t0; a.win_x0 = p->window_x0; a.win_v = p->window_v;
  a.dt_r = (R)p->dt; a.win_v_r = (R)p->window_v;
  a.seed = p->seed; a.scenario = p->scenario; a.step = p->step;
  a.emit = 1; a.pairs = 0; a.drain = 1; a.recoil_energy = p->recoil_energy ? 1 : 0;
  a.ledger_part = reinterpret_cast<double*>(base + kOffLedger);
  a.ledger = a.ledger_part + kMaxGrid * kLedgerN;
  a.plan = reinterpret_cast<FinalizePlan*>(base + kOffPlan);
  a.work = reinterpret_cast<unsigned long long*>(base + kOffWork);
  // every call starts from cleared counters and range sums: the array keeps the last call's
  // contents, and an earlier call may have stopped on an error
  cudaMemsetAsync(ranges, 0, 2 * kRanges * 4, s);
  noalloc_begin_kernel<<<1, 1, 0, s>>>(cnt, (uint32_t)n, counter);
  const int grid = std::min(step_grid_size(sizeof(R) == 4 ? QED_MIXED : QED_FP64), (int)kMaxGrid);
  launch_step<R>(a, grid, 256, 0, s);
  launch_finalize<R>(a, grid, s);
  noalloc_end_kernel<<<1, 1, 0, s>>>(cnt, counter);
  count_launch(2);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return set_error(QED_ERR_CUDA, cudaGetErrorString(err));
  return QED_OK;
}

}  // namespace

extern "C" qed_status qed_step_emit_noalloc(const qed_tables* tables, qed_precision precision,
                                            const qed_soa* electrons, size_t n_electrons, const qed_soa* photons,
                                            size_t photon_capacity, uint32_t* photon_counter,
                                            const qed_step_params* params, void* stream) {
  if (!tables || !electrons || !photons || !photon_counter || !params)
    return set_error(QED_ERR_INVALID_ARG, "qed_step_emit_noalloc: NULL argument");
  if (precision != QED_FP64 && precision != QED_MIXED)
    return set_error(QED_ERR_INVALID_ARG, "qed_step_emit_noalloc: bad precision");
  if (n_electrons > kMaxElectrons)
    return set_error(QED_ERR_INVALID_ARG,
                        "qed_step_emit_noalloc: at most 65536 electrons per call (fixed scratch size)");
  if (photon_capacity > 0x7fffffe0u) return set_error(QED_ERR_INVALID_ARG, "qed_step_emit_noalloc: capacity");
  if (!(params->dt > 0.0) || !std::isfinite(params->dt))
    return set_error(QED_ERR_INVALID_ARG, "qed_step_emit_noalloc: dt must be finite and > 0");
  const qed_status fs = check_field(params->field, "qed_step_emit_noalloc");
  if (fs != QED_OK) return fs;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 128) return set_error(QED_ERR_CUDA, "qed_step_emit_noalloc: no device");
  void* base = nullptr;
  {
    // one-time set-up per device (this device is current): the scratch's device address
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        return set_error(QED_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    base = g_addr[dev];
  }
  // the TMA tile copies need 16-byte aligned arrays
  const void* arrays[16] = {electrons->x, electrons->y, electrons->z, electrons->ux, electrons->uy, electrons->uz,
                            electrons->tau, electrons->id, photons->x, photons->y, photons->z, photons->ux,
                            photons->uy, photons->uz, photons->tau, photons->id};
  for (const void* q : arrays)
    if (n_electrons && (!q || (reinterpret_cast<uintptr_t>(q) & 15u)))
      return set_error(QED_ERR_INVALID_ARG, "qed_step_emit_noalloc: arrays must be non-NULL and 16-byte aligned");
  const TablesDev tv = tables_dev(tables);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* b = static_cast<unsigned char*>(base);
  return precision == QED_MIXED ? run_noalloc<float>(tv, electrons, n_electrons, photons, photon_capacity,
                                                     photon_counter, params, b, s)
                                : run_noalloc<double>(tv, electrons, n_electrons, photons, photon_capacity,
                                                      photon_counter, params, b, s);
}
