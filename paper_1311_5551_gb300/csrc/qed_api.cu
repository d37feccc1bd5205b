// qed_api.cu -- the C ABI of include/qed.h: object lifetimes, device memory through the
// caller's allocator, host <-> device transfers and the launch sequence of one step.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qed_internal.h"

namespace qedlib {
uint64_t launch_count_value();
}

using namespace qedlib;

namespace {

thread_local std::string g_err;
constexpr int kTotalsBlocks = 456;  // blocks (and FP64 partials) of qed_species_totals

// NVTX range around an entry point (visible in a profiler's timeline; near-free otherwise).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

qed_status fail(qed_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

qed_status cuda_fail(cudaError_t e, const char* what) {
  return fail(QED_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define QED_CUDA(call)                                          \
  do {                                                          \
    cudaError_t e__ = (call);                                   \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call);       \
  } while (0)

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Device -> host read on the caller's stream (every call that returns device values synchronises
// that stream, not the device).
cudaError_t read_on(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

// ------------------------------------------------------------------ device memory
struct DeviceBlock {
  qed_allocator alloc{};
  bool have_alloc = false;
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;

  qed_status get(size_t n, const qed_allocator* a, cudaStream_t s) {
    stream = s;
    bytes = n;
    if (a && a->alloc) {
      alloc = *a;
      have_alloc = true;
      ptr = a->alloc(n, (void*)s, a->user);
      if (!ptr) return fail(QED_ERR_OOM, "allocator returned NULL for " + std::to_string(n) + " bytes");
    } else {
      cudaError_t e = cudaMallocAsync(&ptr, n, s);
      if (e != cudaSuccess) { ptr = nullptr; return cuda_fail(e, "cudaMallocAsync"); }
    }
    return QED_OK;
  }
  void release() {
    if (!ptr) return;
    if (have_alloc) {
      if (alloc.free) alloc.free(ptr, bytes, (void*)stream, alloc.user);
    } else {
      cudaFreeAsync(ptr, stream);
    }
    ptr = nullptr;
  }
};

// Carves aligned sub-buffers out of one allocation.
struct Carver {
  size_t off = 0;
  std::vector<std::pair<void**, size_t>> items;
  template <typename T>
  void add(T** p, size_t count) {
    off = (off + 255) & ~size_t(255);
    items.push_back({reinterpret_cast<void**>(p), off});
    off += count * sizeof(T) + 16;
  }
  size_t total() const { return (off + 255) & ~size_t(255); }
  void bind(void* base) {
    for (auto& it : items) *it.first = static_cast<char*>(base) + it.second;
  }
};

__global__ void set_counters_kernel(DevCounters* c, uint32_t n, uint32_t next_id) {
  c->n = n;
  c->next_id = next_id;
  c->n_app = 0;
  c->n_dead = 0;
}
__global__ void iota_kernel(uint32_t* id, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    id[i] = (uint32_t)i;
}

}  // namespace

// ============================================================================ tables
struct qed_tables {
  TableHost host;
  DeviceBlock mem;
  TabDev<double> d64{};
  TabDev<float> d32{};
};

namespace {
template <typename R>
void set_tab_scalars(TabDev<R>& t, const TableHost& h) {
  const qed_table_params& p = h.p;
  t.n_eta = p.n_eta; t.n_xi = p.n_xi; t.n_chi = p.n_chi; t.n_f = p.n_f;
  const double le0 = std::log(p.eta_min), le1 = std::log(p.eta_max);
  const double lc0 = std::log(p.chi_min), lc1 = std::log(p.chi_max);
  t.ln_eta_min = (R)le0;
  t.inv_d_eta = (R)((p.n_eta - 1) / (le1 - le0));
  t.eta_min = (R)p.eta_min;
  t.ln_chi_min = (R)lc0;
  t.inv_d_chi = (R)((p.n_chi - 1) / (lc1 - lc0));
  t.chi_min = (R)p.chi_min;
  t.chi_max = (R)p.chi_max;
  t.T_at_chi_max = (R)std::exp(h.ln_T[p.n_chi - 1]);
}

template <typename R>
void fill_image(std::vector<R>& img, const TableHost& h) {
  img.clear();
  auto put = [&](const std::vector<double>& v) { for (double x : v) img.push_back((R)x); };
  put(h.ln_h); put(h.ln_T); put(h.P); put(h.Q); put(h.zeta_lo); put(h.zeta_hi); put(h.Pf);
}

template <typename R>
void bind_image(TabDev<R>& t, const R* base, const TableHost& h) {
  const R* p = base;
  t.ln_h = p; p += h.ln_h.size();
  t.ln_T = p; p += h.ln_T.size();
  t.P = p; p += h.P.size();
  t.Q = p; p += h.Q.size();
  t.zeta_lo = p; p += h.zeta_lo.size();
  t.zeta_hi = p; p += h.zeta_hi.size();
  t.Pf = p;
}

qed_status upload_tables(qed_tables* T, const qed_allocator* alloc, cudaStream_t s) {
  if (T->host.p.n_eta > 4096 || T->host.p.n_chi > 4096)
    return fail(QED_ERR_INVALID_ARG, "n_eta and n_chi must be <= 4096 (h and T are staged in shared memory)");
  std::vector<double> i64;
  std::vector<float> i32;
  fill_image(i64, T->host);
  fill_image(i32, T->host);
  const size_t b64 = (i64.size() * 8 + 255) & ~size_t(255);
  const size_t b32 = i32.size() * 4;
  qed_status st = T->mem.get(b64 + b32, alloc, s);
  if (st != QED_OK) return st;
  char* base = static_cast<char*>(T->mem.ptr);
  QED_CUDA(cudaMemcpyAsync(base, i64.data(), i64.size() * 8, cudaMemcpyHostToDevice, s));
  QED_CUDA(cudaMemcpyAsync(base + b64, i32.data(), i32.size() * 4, cudaMemcpyHostToDevice, s));
  QED_CUDA(cudaStreamSynchronize(s));  // the host images are locals
  bind_image(T->d64, reinterpret_cast<const double*>(base), T->host);
  bind_image(T->d32, reinterpret_cast<const float*>(base + b64), T->host);
  set_tab_scalars(T->d64, T->host);
  set_tab_scalars(T->d32, T->host);
  return QED_OK;
}
}  // namespace

namespace qedlib {
TablesDev tables_dev(const qed_tables* t) { return TablesDev{t->d64, t->d32}; }
qed_status set_error(qed_status st, const std::string& msg) { return fail(st, msg); }
}  // namespace qedlib

extern "C" qed_status qed_tables_build(const qed_table_params* params, const qed_allocator* alloc, void* stream,
                                       qed_tables** out) {
  if (!params || !out) return fail(QED_ERR_INVALID_ARG, "qed_tables_build: NULL argument");
  *out = nullptr;
  auto* T = new qed_tables();
  std::string err;
  if (!build_tables_host(*params, T->host, err)) { delete T; return fail(QED_ERR_INVALID_ARG, err); }
  qed_status st = upload_tables(T, alloc, as_stream(stream));
  if (st != QED_OK) { T->mem.release(); delete T; return st; }
  *out = T;
  return QED_OK;
}

extern "C" qed_status qed_tables_from_arrays(const qed_table_params* params, const qed_table_arrays* a,
                                             const qed_allocator* alloc, void* stream, qed_tables** out) {
  if (!params || !a || !out) return fail(QED_ERR_INVALID_ARG, "qed_tables_from_arrays: NULL argument");
  *out = nullptr;
  std::string err;
  if (!validate_table_params(*params, err)) return fail(QED_ERR_INVALID_ARG, err);
  if (!a->ln_h || !a->zeta_lo || !a->zeta_hi || !a->P || !a->Q || !a->ln_T || !a->Pf)
    return fail(QED_ERR_INVALID_ARG, "qed_tables_from_arrays: NULL table array");
  auto* T = new qed_tables();
  T->host.resize(*params);
  auto cp = [](std::vector<double>& v, const double* src) { if (src) std::copy(src, src + v.size(), v.begin()); };
  cp(T->host.ln_h, a->ln_h); cp(T->host.g, a->g); cp(T->host.zeta_lo, a->zeta_lo); cp(T->host.zeta_hi, a->zeta_hi);
  cp(T->host.P, a->P); cp(T->host.Q, a->Q); cp(T->host.ln_T, a->ln_T); cp(T->host.Pf, a->Pf);
  qed_status st = upload_tables(T, alloc, as_stream(stream));
  if (st != QED_OK) { T->mem.release(); delete T; return st; }
  *out = T;
  return QED_OK;
}

extern "C" qed_status qed_tables_export(const qed_tables* T, qed_table_arrays* d) {
  if (!T || !d) return fail(QED_ERR_INVALID_ARG, "qed_tables_export: NULL argument");
  auto cp = [](const std::vector<double>& v, double* dst) { if (dst) std::copy(v.begin(), v.end(), dst); };
  cp(T->host.ln_h, d->ln_h); cp(T->host.g, d->g); cp(T->host.zeta_lo, d->zeta_lo); cp(T->host.zeta_hi, d->zeta_hi);
  cp(T->host.P, d->P); cp(T->host.Q, d->Q); cp(T->host.ln_T, d->ln_T); cp(T->host.Pf, d->Pf);
  return QED_OK;
}

extern "C" void qed_tables_free(qed_tables* T) {
  if (!T) return;
  T->mem.release();
  delete T;
}

// ============================================================================ species
struct qed_species {
  int kind = 0, precision = 0;
  size_t cap = 0, acap = 0;
  DeviceBlock mem;
  SpeciesDev<float> f{};
  SpeciesDev<double> d{};
  DevCounters* cnt = nullptr;
  // step workspace (used when this species is passed as sp[0])
  double* ledger_part = nullptr;
  double* ledger = nullptr;
  FinalizePlan* plan = nullptr;
  unsigned long long* work = nullptr;
  uint32_t* first_event = nullptr;  // multi-step probe result
  double* totals_part = nullptr;     // qed_species_totals: per-block partials
  int ledger_parts = 0;
  // macroparticle weights (the species' w and aw arrays), allocated when first needed
  DeviceBlock wmem;
  // second array set for compaction (allocated at the first compaction)
  DeviceBlock alt_mem, alt_wmem;
  qed_allocator alloc_copy{};
  bool have_alloc = false;
  void* other[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* other_tau = nullptr;
  uint32_t* other_id = nullptr;
  void* other_w = nullptr;
  uint32_t* seg_count = nullptr;
  uint32_t* seg_prefix = nullptr;
  int last_drain = 0;
};

namespace {
template <typename R>
void carve_species(Carver& cv, SpeciesDev<R>& s, size_t cap, size_t acap, size_t words, size_t ranges) {
  cv.add(&s.x, cap); cv.add(&s.y, cap); cv.add(&s.z, cap);
  cv.add(&s.ux, cap); cv.add(&s.uy, cap); cv.add(&s.uz, cap);
  cv.add(&s.tau, cap); cv.add(&s.id, cap);
  cv.add(&s.evmask, words); cv.add(&s.wprefix, words);
  cv.add(&s.rangesum, ranges); cv.add(&s.rprefix, ranges);
  cv.add(&s.ax, acap); cv.add(&s.ay, acap); cv.add(&s.az, acap);
  cv.add(&s.aux, acap); cv.add(&s.auy, acap); cv.add(&s.auz, acap);
  cv.add(&s.atau, acap); cv.add(&s.aparent, acap);
}

template <typename R>
qed_soa soa_of(const SpeciesDev<R>& s) {
  qed_soa o;
  o.x = s.x; o.y = s.y; o.z = s.z; o.ux = s.ux; o.uy = s.uy; o.uz = s.uz; o.tau = s.tau; o.id = s.id;
  return o;
}
size_t elem_bytes(const qed_species* sp) { return sp->precision == QED_MIXED ? 4 : 8; }
qed_soa soa(const qed_species* sp) { return sp->precision == QED_MIXED ? soa_of(sp->f) : soa_of(sp->d); }

qed_status read_counters(const qed_species* sp, DevCounters& c, cudaStream_t s) {
  QED_CUDA(read_on(&c, sp->cnt, sizeof(DevCounters), s));
  return QED_OK;
}

bool has_weights(const qed_species* sp) { return sp->precision == QED_MIXED ? sp->f.w != nullptr : sp->d.w != nullptr; }
void* weights_of(const qed_species* sp) {
  return sp->precision == QED_MIXED ? (void*)sp->f.w : (void*)sp->d.w;
}

// Weights are optional: a species without a weight array stands for weight 1 per particle (the
// step reads weights only at events, to hand them to the children).  The arrays (held particles
// and append region) are allocated, through the species' allocator, the first time weights are
// set, merged, restored or needed because a partner species of a step has them; they start at 1.
template <typename R>
qed_status ensure_weights_t(qed_species* sp, SpeciesDev<R>& d, cudaStream_t s) {
  if (d.w) return QED_OK;
  const size_t cap = sp->cap, acap = std::max<size_t>(sp->acap, 1);
  const size_t off = ((cap * sizeof(R)) + 255) & ~size_t(255);
  qed_status st = sp->wmem.get(off + acap * sizeof(R), sp->have_alloc ? &sp->alloc_copy : nullptr, s);
  if (st != QED_OK) return st;
  d.w = static_cast<R*>(sp->wmem.ptr);
  d.aw = reinterpret_cast<R*>(static_cast<char*>(sp->wmem.ptr) + off);
  launch_fill<R>(d.w, cap, (R)1, s);
  launch_fill<R>(d.aw, acap, (R)1, s);
  QED_CUDA(cudaGetLastError());
  return QED_OK;
}
qed_status ensure_weights(qed_species* sp, cudaStream_t s) {
  return sp->precision == QED_MIXED ? ensure_weights_t(sp, sp->f, s) : ensure_weights_t(sp, sp->d, s);
}
// Children inherit their parent's weight: when any species of a step holds weights, all of them
// (and the drain) get weight arrays, so no child loses its parent's weight.
qed_status sync_weights(qed_species* const* sp, cudaStream_t s) {
  bool any = false;
  for (int k = 0; k < 4; ++k) any |= sp[k] && has_weights(sp[k]);
  if (!any) return QED_OK;
  for (int k = 0; k < 4; ++k)
    if (sp[k]) { qed_status st = ensure_weights(sp[k], s); if (st != QED_OK) return st; }
  return QED_OK;
}

// n values of 1 in the species precision at dst, host or device memory.
qed_status write_ones(void* dst, size_t n, int precision, cudaStream_t s) {
  if (!n) return QED_OK;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, dst) == cudaSuccess &&
      (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
    if (precision == QED_MIXED) launch_fill<float>(static_cast<float*>(dst), n, 1.0f, s);
    else launch_fill<double>(static_cast<double*>(dst), n, 1.0, s);
    QED_CUDA(cudaGetLastError());
    return QED_OK;
  }
  cudaGetLastError();  // a host pointer unknown to CUDA is not an error here
  QED_CUDA(cudaStreamSynchronize(s));  // earlier copies into dst are done
  if (precision == QED_MIXED) std::fill(static_cast<float*>(dst), static_cast<float*>(dst) + n, 1.0f);
  else std::fill(static_cast<double*>(dst), static_cast<double*>(dst) + n, 1.0);
  return QED_OK;
}
}  // namespace

extern "C" qed_status qed_species_alloc(qed_kind kind, qed_precision precision, size_t capacity,
                                        size_t append_capacity, const qed_allocator* alloc, void* stream,
                                        qed_species** out) {
  if (!out) return fail(QED_ERR_INVALID_ARG, "qed_species_alloc: NULL out");
  *out = nullptr;
  if (kind < QED_ELECTRON || kind > QED_PHOTON) return fail(QED_ERR_INVALID_ARG, "bad species kind");
  if (precision != QED_FP64 && precision != QED_MIXED) return fail(QED_ERR_INVALID_ARG, "bad precision");
  if (capacity == 0 || capacity > 0x7fffffe0u || append_capacity > 0x7fffffe0u)
    return fail(QED_ERR_INVALID_ARG, "capacity must be in [1, 2^31 - 32]");
  cudaStream_t s = as_stream(stream);
  auto* sp = new qed_species();
  sp->kind = kind;
  sp->precision = precision;
  sp->cap = capacity;
  sp->acap = append_capacity;
  const size_t words = capacity / 32 + 2;
  const size_t ranges = (words >> kRangeShift) + 2;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sp->ledger_parts = std::max(step_grid_size(QED_MIXED), step_grid_size(QED_FP64));
  Carver cv;
  if (precision == QED_MIXED) carve_species(cv, sp->f, capacity, std::max<size_t>(append_capacity, 1), words, ranges);
  else carve_species(cv, sp->d, capacity, std::max<size_t>(append_capacity, 1), words, ranges);
  cv.add(&sp->cnt, 1);
  cv.add(&sp->ledger_part, (size_t)sp->ledger_parts * kLedgerN);
  cv.add(&sp->ledger, kLedgerN);
  cv.add(&sp->plan, 1);
  cv.add(&sp->work, 6);
  cv.add(&sp->first_event, 1);
  cv.add(&sp->totals_part, (size_t)kTotalsBlocks * 5);
  qed_status st = sp->mem.get(cv.total(), alloc, s);
  if (st != QED_OK) { delete sp; return st; }
  cv.bind(sp->mem.ptr);
  if (alloc && alloc->alloc) { sp->alloc_copy = *alloc; sp->have_alloc = true; }
  cudaError_t e = cudaMemsetAsync(sp->mem.ptr, 0, cv.total(), s);
  if (e != cudaSuccess) { sp->mem.release(); delete sp; return cuda_fail(e, "cudaMemsetAsync"); }
  auto fill = [&](auto& S) {
    S.cap = (uint32_t)capacity;
    S.acap = (uint32_t)append_capacity;
    S.cnt = sp->cnt;
  };
  if (precision == QED_MIXED) fill(sp->f); else fill(sp->d);
  *out = sp;
  return QED_OK;
}

extern "C" void qed_species_free(qed_species* sp) {
  if (!sp) return;
  sp->alt_wmem.release();
  sp->alt_mem.release();
  sp->wmem.release();
  sp->mem.release();
  delete sp;
}

extern "C" qed_status qed_species_upload(qed_species* sp, const qed_soa* src, size_t n, uint32_t next_id,
                                         void* stream) {
  if (!sp || !src) return fail(QED_ERR_INVALID_ARG, "qed_species_upload: NULL argument");
  if (n > sp->cap) return fail(QED_ERR_CAPACITY, "qed_species_upload: n exceeds capacity");
  if (n > 0 && (!src->x || !src->y || !src->z || !src->ux || !src->uy || !src->uz))
    return fail(QED_ERR_INVALID_ARG, "qed_species_upload: NULL position or momentum array");
  cudaStream_t s = as_stream(stream);
  const qed_soa d = soa(sp);
  const size_t b = elem_bytes(sp) * n;
  if (n > 0) {
    QED_CUDA(cudaMemcpyAsync(d.x, src->x, b, cudaMemcpyDefault, s));
    QED_CUDA(cudaMemcpyAsync(d.y, src->y, b, cudaMemcpyDefault, s));
    QED_CUDA(cudaMemcpyAsync(d.z, src->z, b, cudaMemcpyDefault, s));
    QED_CUDA(cudaMemcpyAsync(d.ux, src->ux, b, cudaMemcpyDefault, s));
    QED_CUDA(cudaMemcpyAsync(d.uy, src->uy, b, cudaMemcpyDefault, s));
    QED_CUDA(cudaMemcpyAsync(d.uz, src->uz, b, cudaMemcpyDefault, s));
    if (src->tau) {
      QED_CUDA(cudaMemcpyAsync(d.tau, src->tau, 8 * n, cudaMemcpyDefault, s));
      launch_tau_convert(sp->precision, d.tau, n, false, s);  // double -> stored form
    } else {
      QED_CUDA(cudaMemsetAsync(d.tau, 0, 8 * n, s));  // zero in either form
    }
    if (src->id) {
      QED_CUDA(cudaMemcpyAsync(d.id, src->id, 4 * n, cudaMemcpyDefault, s));
    } else {
      iota_kernel<<<64, 256, 0, s>>>(d.id, n);
      count_launch();
    }
  }
  // weights (if the species has them): 1, until qed_species_set_weights
  if (has_weights(sp)) {
    if (sp->precision == QED_MIXED) launch_fill<float>(sp->f.w, n, 1.0f, s);
    else launch_fill<double>(sp->d.w, n, 1.0, s);
  }
  const uint32_t nid = src->id ? next_id : (uint32_t)n;
  set_counters_kernel<<<1, 1, 0, s>>>(sp->cnt, (uint32_t)n, nid);
  count_launch();
  QED_CUDA(cudaGetLastError());
  return QED_OK;
}

extern "C" qed_status qed_species_download(qed_species* sp, const qed_soa* dst, size_t cap, size_t* n_out,
                                           void* stream) {
  if (!sp || !dst || !n_out) return fail(QED_ERR_INVALID_ARG, "qed_species_download: NULL argument");
  cudaStream_t s = as_stream(stream);
  DevCounters c;
  qed_status st = read_counters(sp, c, s);
  if (st != QED_OK) return st;
  const size_t n = std::min<size_t>(c.n, cap);
  const qed_soa d = soa(sp);
  const size_t b = elem_bytes(sp) * n;
  if (n > 0) {
    if (dst->x) QED_CUDA(cudaMemcpyAsync(dst->x, d.x, b, cudaMemcpyDefault, s));
    if (dst->y) QED_CUDA(cudaMemcpyAsync(dst->y, d.y, b, cudaMemcpyDefault, s));
    if (dst->z) QED_CUDA(cudaMemcpyAsync(dst->z, d.z, b, cudaMemcpyDefault, s));
    if (dst->ux) QED_CUDA(cudaMemcpyAsync(dst->ux, d.ux, b, cudaMemcpyDefault, s));
    if (dst->uy) QED_CUDA(cudaMemcpyAsync(dst->uy, d.uy, b, cudaMemcpyDefault, s));
    if (dst->uz) QED_CUDA(cudaMemcpyAsync(dst->uz, d.uz, b, cudaMemcpyDefault, s));
    if (dst->tau) {
      // the stored form becomes double for the copy and is restored afterwards (exact round trip)
      launch_tau_convert(sp->precision, d.tau, n, true, s);
      QED_CUDA(cudaMemcpyAsync(dst->tau, d.tau, 8 * n, cudaMemcpyDefault, s));
      launch_tau_convert(sp->precision, d.tau, n, false, s);
    }
    if (dst->id) QED_CUDA(cudaMemcpyAsync(dst->id, d.id, 4 * n, cudaMemcpyDefault, s));
  }
  QED_CUDA(cudaStreamSynchronize(s));
  *n_out = c.n;
  if (c.err) return fail(QED_ERR_CAPACITY, "device error flags set on species (see qed_check)");
  return QED_OK;
}

extern "C" qed_status qed_species_count(const qed_species* sp, size_t* n_out, void* stream) {
  if (!sp || !n_out) return fail(QED_ERR_INVALID_ARG, "qed_species_count: NULL argument");
  DevCounters c;
  qed_status st = read_counters(sp, c, as_stream(stream));
  if (st != QED_OK) return st;
  *n_out = c.n;
  return QED_OK;
}

extern "C" qed_status qed_species_view_get(const qed_species* sp, qed_species_view* v) {
  if (!sp || !v) return fail(QED_ERR_INVALID_ARG, "qed_species_view_get: NULL argument");
  v->arrays = soa(sp);
  v->capacity = sp->cap;
  v->kind = sp->kind;
  v->precision = sp->precision;
  return QED_OK;
}

namespace {
struct CheckpointHeader {
  uint32_t magic, version;
  int32_t kind, precision;
  uint64_t n;
  uint32_t next_id, n_dead;
  uint8_t pad[32];
};
static_assert(sizeof(CheckpointHeader) == 64, "checkpoint header is 64 bytes");
constexpr uint32_t kCkptMagic = 0x51454443u;  // "CDEQ"

size_t checkpoint_bytes(const qed_species* sp, size_t n) {
  return sizeof(CheckpointHeader) + n * (7 * elem_bytes(sp) + 8 + 4);
}
constexpr int kCkptHasWeights = 0;  // pad byte: 1 when the species held a weight array

__global__ void set_counters_full_kernel(DevCounters* c, uint32_t n, uint32_t next_id, uint32_t n_dead) {
  c->n = n;
  c->next_id = next_id;
  c->n_app = 0;
  c->n_dead = n_dead;
}
}  // namespace

extern "C" qed_status qed_species_save(qed_species* sp, void* dst, size_t cap_bytes, size_t* bytes_out,
                                       void* stream) {
  if (!sp || !bytes_out) return fail(QED_ERR_INVALID_ARG, "qed_species_save: NULL argument");
  cudaStream_t s = as_stream(stream);
  DevCounters c;
  qed_status st = read_counters(sp, c, s);
  if (st != QED_OK) return st;
  const size_t need = checkpoint_bytes(sp, c.n);
  *bytes_out = need;
  if (!dst) return QED_OK;
  if (cap_bytes < need) return fail(QED_ERR_CAPACITY, "qed_species_save: destination too small");
  CheckpointHeader h{};
  h.magic = kCkptMagic; h.version = 2; h.kind = sp->kind; h.precision = sp->precision;
  h.n = c.n; h.next_id = c.next_id; h.n_dead = c.n_dead;
  h.pad[kCkptHasWeights] = has_weights(sp) ? 1 : 0;
  char* out = static_cast<char*>(dst);
  QED_CUDA(cudaMemcpyAsync(out, &h, sizeof(h), cudaMemcpyDefault, s));
  const qed_soa d = soa(sp);
  const size_t b = elem_bytes(sp) * c.n;
  size_t off = sizeof(h);
  for (void* a : {d.x, d.y, d.z, d.ux, d.uy, d.uz}) { QED_CUDA(cudaMemcpyAsync(out + off, a, b, cudaMemcpyDefault, s)); off += b; }
  QED_CUDA(cudaMemcpyAsync(out + off, d.tau, 8 * c.n, cudaMemcpyDefault, s)); off += 8 * c.n;
  QED_CUDA(cudaMemcpyAsync(out + off, d.id, 4 * c.n, cudaMemcpyDefault, s)); off += 4 * c.n;
  if (has_weights(sp)) {
    QED_CUDA(cudaMemcpyAsync(out + off, weights_of(sp), b, cudaMemcpyDefault, s));
  } else {
    qed_status wst = write_ones(out + off, c.n, sp->precision, s);
    if (wst != QED_OK) return wst;
  }
  QED_CUDA(cudaStreamSynchronize(s));  // the header is a local
  return QED_OK;
}

extern "C" qed_status qed_species_restore(qed_species* sp, const void* src, size_t bytes, void* stream) {
  if (!sp || !src) return fail(QED_ERR_INVALID_ARG, "qed_species_restore: NULL argument");
  if (bytes < sizeof(CheckpointHeader)) return fail(QED_ERR_INVALID_ARG, "qed_species_restore: truncated checkpoint");
  cudaStream_t s = as_stream(stream);
  CheckpointHeader h;
  QED_CUDA(read_on(&h, src, sizeof(h), s));
  if (h.magic != kCkptMagic || h.version != 2) return fail(QED_ERR_INVALID_ARG, "qed_species_restore: not a checkpoint");
  if (h.kind != sp->kind || h.precision != sp->precision)
    return fail(QED_ERR_INVALID_ARG, "qed_species_restore: kind or precision differs");
  if (h.n > sp->cap) return fail(QED_ERR_CAPACITY, "qed_species_restore: checkpoint exceeds capacity");
  if (bytes < checkpoint_bytes(sp, h.n)) return fail(QED_ERR_INVALID_ARG, "qed_species_restore: truncated checkpoint");
  const char* in = static_cast<const char*>(src);
  const qed_soa d = soa(sp);
  const size_t b = elem_bytes(sp) * h.n;
  size_t off = sizeof(h);
  for (void* a : {d.x, d.y, d.z, d.ux, d.uy, d.uz}) { QED_CUDA(cudaMemcpyAsync(a, in + off, b, cudaMemcpyDefault, s)); off += b; }
  QED_CUDA(cudaMemcpyAsync(d.tau, in + off, 8 * h.n, cudaMemcpyDefault, s)); off += 8 * h.n;
  QED_CUDA(cudaMemcpyAsync(d.id, in + off, 4 * h.n, cudaMemcpyDefault, s)); off += 4 * h.n;
  if (h.pad[kCkptHasWeights]) {
    qed_status wst = ensure_weights(sp, s);
    if (wst != QED_OK) return wst;
    QED_CUDA(cudaMemcpyAsync(weights_of(sp), in + off, b, cudaMemcpyDefault, s));
  } else if (has_weights(sp)) {
    if (sp->precision == QED_MIXED) launch_fill<float>(sp->f.w, h.n, 1.0f, s);
    else launch_fill<double>(sp->d.w, h.n, 1.0, s);
  }
  set_counters_full_kernel<<<1, 1, 0, s>>>(sp->cnt, (uint32_t)h.n, h.next_id, h.n_dead);
  count_launch();
  QED_CUDA(cudaGetLastError());
  return QED_OK;
}

extern "C" qed_status qed_species_init_tau(qed_species* sp, uint64_t seed, uint64_t scenario, void* stream) {
  if (!sp) return fail(QED_ERR_INVALID_ARG, "qed_species_init_tau: NULL species");
  cudaStream_t s = as_stream(stream);
  if (sp->precision == QED_MIXED) launch_init_tau(sp->f, sp->kind, seed, scenario, s);
  else launch_init_tau(sp->d, sp->kind, seed, scenario, s);
  QED_CUDA(cudaGetLastError());
  return QED_OK;
}

namespace {
// Ping-pong compaction: the survivors are written, in order, into the other array set, which
// then becomes the species' arrays.  The second set (and the scan scratch) is allocated at the
// first compaction.
template <typename R>
qed_status compact_impl(qed_species* sp, SpeciesDev<R>& cur, cudaStream_t s) {
  const size_t cap = sp->cap, segs = cap / 2048 + 2;
  if (!sp->alt_mem.ptr) {
    Carver cv;
    SpeciesDev<R> b = cur;
    cv.add(&b.x, cap); cv.add(&b.y, cap); cv.add(&b.z, cap); cv.add(&b.ux, cap); cv.add(&b.uy, cap);
    cv.add(&b.uz, cap); cv.add(&b.tau, cap); cv.add(&b.id, cap);
    cv.add(&sp->seg_count, segs); cv.add(&sp->seg_prefix, segs + 1);
    qed_status st = sp->alt_mem.get(cv.total(), sp->have_alloc ? &sp->alloc_copy : nullptr, s);
    if (st != QED_OK) return st;
    cv.bind(sp->alt_mem.ptr);
    sp->other[0] = b.x; sp->other[1] = b.y; sp->other[2] = b.z;
    sp->other[3] = b.ux; sp->other[4] = b.uy; sp->other[5] = b.uz;
    sp->other_tau = b.tau; sp->other_id = b.id;
  }
  if (cur.w && !sp->other_w) {  // the second set's weights, once the species has weights
    qed_status st = sp->alt_wmem.get(cap * sizeof(R), sp->have_alloc ? &sp->alloc_copy : nullptr, s);
    if (st != QED_OK) return st;
    sp->other_w = sp->alt_wmem.ptr;
  }
  SpeciesDev<R> out = cur;
  out.x = (R*)sp->other[0]; out.y = (R*)sp->other[1]; out.z = (R*)sp->other[2];
  out.ux = (R*)sp->other[3]; out.uy = (R*)sp->other[4]; out.uz = (R*)sp->other[5];
  out.tau = sp->other_tau; out.id = sp->other_id; out.w = (R*)sp->other_w;
  launch_compact<R>(cur, out, sp->seg_count, sp->seg_prefix, s);
  QED_CUDA(cudaGetLastError());
  // swap the two sets
  sp->other[0] = cur.x; sp->other[1] = cur.y; sp->other[2] = cur.z;
  sp->other[3] = cur.ux; sp->other[4] = cur.uy; sp->other[5] = cur.uz;
  sp->other_tau = cur.tau; sp->other_id = cur.id; sp->other_w = cur.w;
  cur.x = out.x; cur.y = out.y; cur.z = out.z; cur.ux = out.ux; cur.uy = out.uy; cur.uz = out.uz;
  cur.tau = out.tau; cur.id = out.id; cur.w = out.w;
  return QED_OK;
}
}  // namespace

extern "C" qed_status qed_species_compact(qed_species* sp, void* stream) {
  if (!sp) return fail(QED_ERR_INVALID_ARG, "qed_species_compact: NULL species");
  cudaStream_t s = as_stream(stream);
  return sp->precision == QED_MIXED ? compact_impl(sp, sp->f, s) : compact_impl(sp, sp->d, s);
}

extern "C" qed_status qed_species_set_weights(qed_species* sp, const void* w, size_t n, void* stream) {
  if (!sp || (n && !w)) return fail(QED_ERR_INVALID_ARG, "qed_species_set_weights: NULL argument");
  if (n > sp->cap) return fail(QED_ERR_CAPACITY, "qed_species_set_weights: n exceeds capacity");
  cudaStream_t s = as_stream(stream);
  qed_status st = ensure_weights(sp, s);
  if (st != QED_OK) return st;
  if (n) QED_CUDA(cudaMemcpyAsync(weights_of(sp), w, n * elem_bytes(sp), cudaMemcpyDefault, s));
  return QED_OK;
}

extern "C" qed_status qed_species_get_weights(qed_species* sp, void* dst, size_t cap, size_t* n_out, void* stream) {
  if (!sp || !dst || !n_out) return fail(QED_ERR_INVALID_ARG, "qed_species_get_weights: NULL argument");
  cudaStream_t s = as_stream(stream);
  DevCounters c;
  qed_status st = read_counters(sp, c, s);
  if (st != QED_OK) return st;
  const size_t n = std::min<size_t>(c.n, cap);
  if (!has_weights(sp)) {
    st = write_ones(dst, n, sp->precision, s);
    if (st != QED_OK) return st;
  } else if (n) {
    QED_CUDA(cudaMemcpyAsync(dst, weights_of(sp), n * elem_bytes(sp), cudaMemcpyDefault, s));
  }
  QED_CUDA(cudaStreamSynchronize(s));
  *n_out = n;
  return QED_OK;
}

extern "C" qed_status qed_species_totals(qed_species* sp, double out[5], void* stream) {
  if (!sp || !out) return fail(QED_ERR_INVALID_ARG, "qed_species_totals: NULL argument");
  cudaStream_t s = as_stream(stream);
  const int blocks = kTotalsBlocks;
  double* d = sp->totals_part;  // carved out of the species' own allocation
  const int massless = sp->kind == QED_PHOTON ? 1 : 0;
  if (sp->precision == QED_MIXED) launch_totals<float>(sp->f, massless, d, blocks, s);
  else launch_totals<double>(sp->d, massless, d, blocks, s);
  std::vector<double> h(5 * blocks);
  QED_CUDA(read_on(h.data(), d, sizeof(double) * h.size(), s));
  for (int c = 0; c < 5; ++c) out[c] = 0.0;
  for (int b = 0; b < blocks; ++b)
    for (int c = 0; c < 5; ++c) out[c] += h[5 * b + c];  // fixed order
  return QED_OK;
}

extern "C" qed_status qed_species_merge(qed_species* sp, const qed_merge_params* m, uint64_t* groups_out,
                                        void* stream) {
  if (!sp || !m || !groups_out) return fail(QED_ERR_INVALID_ARG, "qed_species_merge: NULL argument");
  if (m->n_face < 1 || m->n_sub < 1 || m->min_group < 3)
    return fail(QED_ERR_INVALID_ARG, "qed_species_merge: n_face, n_sub >= 1 and min_group >= 3");
  MergeDev md{};
  uint64_t cells = 1;
  for (int a = 0; a < 3; ++a) {
    if (!(m->cell[a] > 0.0) || !std::isfinite(m->cell[a]) || !std::isfinite(m->origin[a]) || m->n_cells[a] < 1)
      return fail(QED_ERR_INVALID_ARG, "qed_species_merge: cells must be finite, > 0 and at least one per axis");
    cells *= (uint64_t)m->n_cells[a];
    md.origin[a] = m->origin[a]; md.cell[a] = m->cell[a]; md.n_cells[a] = m->n_cells[a];
  }
  if (cells > 0xffffffffull || 6ull * m->n_face * m->n_face > 0xffffull || (uint64_t)m->n_sub * 2200 > 0xffffull)
    return fail(QED_ERR_INVALID_ARG, "qed_species_merge: too many bins for the 64-bit group key");
  md.n_face = m->n_face; md.n_sub = m->n_sub; md.min_group = m->min_group;
  cudaStream_t s = as_stream(stream);
  DevCounters c;
  qed_status st = read_counters(sp, c, s);
  if (st != QED_OK) return st;
  *groups_out = 0;
  if (c.n < 3) return QED_OK;
  st = ensure_weights(sp, s);  // merged particles carry weights other than 1
  if (st != QED_OK) return st;
  uint32_t N = 1;
  while (N < c.n) N <<= 1;
  // sort scratch through the allocator the species was created with (the library does not
  // allocate on its own behalf)
  const size_t bytes = (size_t)N * 12 + 256;
  DeviceBlock scratch;
  st = scratch.get(bytes, sp->have_alloc ? &sp->alloc_copy : nullptr, s);
  if (st != QED_OK) return st;
  char* tmp = static_cast<char*>(scratch.ptr);
  uint64_t* keys = reinterpret_cast<uint64_t*>(tmp);
  uint32_t* idx = reinterpret_cast<uint32_t*>(tmp + (size_t)N * 8);
  unsigned long long* groups = reinterpret_cast<unsigned long long*>(tmp + (size_t)N * 12 + 128);
  cudaError_t e = cudaMemsetAsync(groups, 0, 8, s);
  if (e != cudaSuccess) { scratch.release(); return cuda_fail(e, "cudaMemsetAsync"); }
  const int massless = sp->kind == QED_PHOTON ? 1 : 0;
  if (sp->precision == QED_MIXED) launch_merge<float>(sp->f, md, keys, idx, N, massless, groups, s);
  else launch_merge<double>(sp->d, md, keys, idx, N, massless, groups, s);
  unsigned long long g = 0;
  e = read_on(&g, groups, 8, s);
  scratch.release();  // ordered after the merge kernels on s
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
  *groups_out = g;
  // the merged-away particles are holes now (tau = +inf): remove them, keeping the order
  st = sp->precision == QED_MIXED ? compact_impl(sp, sp->f, s) : compact_impl(sp, sp->d, s);
  if (st != QED_OK) return st;
  QED_CUDA(cudaGetLastError());
  return QED_OK;
}

// ============================================================================ step
namespace {
// Step-kernel timing: a pool of event pairs, recorded around each step-kernel launch while on.
struct TimingPool {
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  size_t used = 0;
};
TimingPool g_timing;        // per-step kernel launches
TimingPool g_timing_multi;  // multi-step passes (probe or commit)

bool timing_events(cudaEvent_t& a, cudaEvent_t& b, TimingPool& P = g_timing) {
  if (!g_timing.on) return false;
  if (P.used == P.ev.size()) {
    cudaEvent_t x, y;
    if (cudaEventCreate(&x) != cudaSuccess) return false;
    if (cudaEventCreate(&y) != cudaSuccess) { cudaEventDestroy(x); return false; }
    P.ev.push_back({x, y});
  }
  a = P.ev[P.used].first;
  b = P.ev[P.used].second;
  ++P.used;
  return true;
}

qed_status timing_sum(TimingPool& P, double* ms, uint64_t* launches, int reset) {
  double total = 0.0;
  for (size_t k = 0; k < P.used; ++k) {
    QED_CUDA(cudaEventSynchronize(P.ev[k].second));
    float t = 0.f;
    QED_CUDA(cudaEventElapsedTime(&t, P.ev[k].first, P.ev[k].second));
    total += t;
  }
  *ms = total;
  *launches = P.used;
  if (reset) P.used = 0;
  return QED_OK;
}


template <typename R> SpeciesDev<R>& dev_of(qed_species* s);
template <> SpeciesDev<float>& dev_of<float>(qed_species* s) { return s->f; }
template <> SpeciesDev<double>& dev_of<double>(qed_species* s) { return s->d; }
template <typename R> const TabDev<R>& tab_of(const qed_tables* t);
template <> const TabDev<float>& tab_of<float>(const qed_tables* t) { return t->d32; }
template <> const TabDev<double>& tab_of<double>(const qed_tables* t) { return t->d64; }

template <typename R>
StepArgs<R> make_args(const qed_tables* T, qed_species* const* sp, const qed_step_params& p, uint64_t step) {
  StepArgs<R> a{};
  for (int k = 0; k < 3; ++k) a.sp[k] = dev_of<R>(sp[k]);
  a.sp[3] = sp[3] ? dev_of<R>(sp[3]) : dev_of<R>(sp[2]);
  a.tab = tab_of<R>(T);
  a.field = field_dev(p.field);
  a.dt = p.dt; a.t0 = p.t0; a.win_x0 = p.window_x0; a.win_v = p.window_v;
  a.dt_r = (R)p.dt; a.win_v_r = (R)p.window_v;
  a.seed = p.seed; a.scenario = p.scenario; a.step = step;
  a.emit = p.emit_photons ? 1 : 0;
  a.pairs = p.make_pairs ? 1 : 0;
  a.drain = p.drain_photons ? 1 : 0;
  a.recoil_energy = p.recoil_energy ? 1 : 0;
  a.ledger_part = sp[0]->ledger_part;
  a.ledger = sp[0]->ledger;
  a.plan = sp[0]->plan;
  a.work = sp[0]->work;
  return a;
}

template <typename R>
qed_status do_step(const qed_tables* T, qed_species* const* sp, const qed_step_params& p, uint64_t step,
                   cudaStream_t s) {
  const StepArgs<R> a = make_args<R>(T, sp, p, step);
  const int grid = std::min(step_grid_size(sizeof(R) == 4 ? QED_MIXED : QED_FP64), sp[0]->ledger_parts);
  const size_t smem = (size_t)(a.tab.n_eta + a.tab.n_chi) * sizeof(R);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool timed = timing_events(e0, e1);
  if (timed) cudaEventRecord(e0, s);
  launch_step<R>(a, grid, 256, smem, s);
  if (timed) cudaEventRecord(e1, s);
  launch_finalize<R>(a, grid, s);
  sp[0]->last_drain = a.drain;
  return QED_OK;
}

qed_status check_step_args(const qed_tables* T, qed_species* const* sp, const qed_step_params* p) {
  if (!T || !sp || !p) return fail(QED_ERR_INVALID_ARG, "qed_step: NULL argument");
  for (int k = 0; k < 3; ++k)
    if (!sp[k]) return fail(QED_ERR_INVALID_ARG, "qed_step: sp[0..2] must be electrons, positrons, photons");
  if (sp[0]->kind != QED_ELECTRON || sp[1]->kind != QED_POSITRON || sp[2]->kind != QED_PHOTON)
    return fail(QED_ERR_INVALID_ARG, "qed_step: species kinds must be (electron, positron, photon)");
  const int prec = sp[0]->precision;
  for (int k = 1; k < 4; ++k)
    if (sp[k] && sp[k]->precision != prec) return fail(QED_ERR_INVALID_ARG, "qed_step: species precisions differ");
  if (p->drain_photons && (!sp[3] || sp[3]->kind != QED_PHOTON))
    return fail(QED_ERR_INVALID_ARG, "qed_step: drain_photons needs a photon drain species in sp[3]");
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return fail(QED_ERR_INVALID_ARG, "qed_step: dt must be finite and > 0");
  return check_field(p->field, "qed_step");
}
}  // namespace

namespace qedlib {
FieldDev field_dev(const qed_field_desc& f) {
  FieldDev d{};
  d.kind = f.kind;
  for (int c = 0; c < 3; ++c) { d.E[c] = f.E[c]; d.B[c] = f.B[c]; }
  d.E0 = f.E0; d.omega = f.omega; d.phase0 = f.phase0; d.phi_start = f.phi_start; d.phi_len = f.phi_len;
  if (f.kind == QED_FIELD_GRID) {
    d.grid = f.grid;
    d.shape = f.shape;
    for (int c = 0; c < 3; ++c) { d.n[c] = f.n[c]; d.origin[c] = f.origin[c]; d.spacing[c] = f.spacing[c]; }
  }
  return d;
}

qed_status check_field(const qed_field_desc& f, const char* who) {
  const std::string w(who);
  if (f.kind < QED_FIELD_UNIFORM || f.kind > QED_FIELD_GRID) return fail(QED_ERR_INVALID_ARG, w + ": unknown field kind");
  for (int c = 0; c < 3; ++c)
    if (!std::isfinite(f.E[c]) || !std::isfinite(f.B[c])) return fail(QED_ERR_NUMERIC, w + ": non-finite field");
  if (!std::isfinite(f.E0) || !std::isfinite(f.omega) || !std::isfinite(f.phi_start) || !std::isfinite(f.phi_len) ||
      !std::isfinite(f.phase0))
    return fail(QED_ERR_NUMERIC, w + ": non-finite field parameter");
  if (f.kind == QED_FIELD_GRID) {
    if (!f.grid) return fail(QED_ERR_INVALID_ARG, w + ": grid field without grid array");
    if (f.shape != 1 && f.shape != 2) return fail(QED_ERR_INVALID_ARG, w + ": grid shape must be 1 (CIC) or 2 (TSC)");
    for (int c = 0; c < 3; ++c) {
      if (f.n[c] < 1) return fail(QED_ERR_INVALID_ARG, w + ": grid needs at least one node per axis");
      if (!(f.spacing[c] > 0.0) || !std::isfinite(f.spacing[c]) || !std::isfinite(f.origin[c]))
        return fail(QED_ERR_INVALID_ARG, w + ": grid spacing must be finite and > 0, origin finite");
    }
  }
  return QED_OK;
}
}  // namespace qedlib

// ============================================================================ batches
struct qed_batch {
  const qed_tables* tables = nullptr;
  int precision = 0, S = 0;
  DeviceBlock mem;
  void* args = nullptr;  // StepArgs<R>[S]
  uint32_t *remaining = nullptr, *live = nullptr, *blocks = nullptr, *first_event = nullptr, *tried = nullptr,
           *skip = nullptr, *span = nullptr, *tot = nullptr;
  SlotPlan* splan = nullptr;
  void* scal = nullptr;  // StepScalars<R>[S]
  int target_blocks = 0, graph_steps = 32, max_parts = 0, fuse_k = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_for_steps = 0, graph_for_target = 0, graph_for_grid = 0, graph_for_fuse = 0;
  std::vector<char> slot_grid;  // slot's field is gathered from a grid
  int grid_fields = 0;
  // graphs are captured on, and replayed from, a stream of the batch's own (the caller's stream
  // may be the legacy default stream, which cannot be captured); events order it with the
  // caller's stream
  cudaStream_t own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace {
template <typename R>
BatchCtl<R> batch_ctl(const qed_batch* b) {
  BatchCtl<R> c;
  c.args = static_cast<StepArgs<R>*>(b->args);
  c.remaining = b->remaining; c.live = b->live; c.blocks = b->blocks;
  c.S = b->S; c.target_blocks = b->target_blocks; c.max_parts = b->max_parts;
  c.grid_fields = b->grid_fields;
  c.first_event = b->first_event;
  c.tried = b->tried;
  c.skip = b->skip;
  c.span = b->span;
  c.fuse_k = b->fuse_k;
  c.splan = b->splan;
  c.scal = b->scal;
  c.tot = b->tot;
  c.tab = tab_of<R>(b->tables);
  return c;
}

void launch_batch(const qed_batch* b, cudaStream_t s) {
  const TableHost& h = b->tables->host;
  if (b->precision == QED_MIXED) launch_batch_step<float>(batch_ctl<float>(b), h.p.n_eta, h.p.n_chi, s);
  else launch_batch_step<double>(batch_ctl<double>(b), h.p.n_eta, h.p.n_chi, s);
}

void set_slot_grid(qed_batch* b, int slot, bool grid) {
  if (b->slot_grid.size() != (size_t)b->S) b->slot_grid.assign(b->S, 0);
  b->slot_grid[slot] = grid ? 1 : 0;
  b->grid_fields = 0;
  for (char g : b->slot_grid) b->grid_fields |= g;
}

void drop_graph(qed_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_for_steps = 0;
}

qed_status ensure_graph(qed_batch* b) {
  if (b->graph && b->graph_for_steps == b->graph_steps && b->graph_for_target == b->target_blocks &&
      b->graph_for_grid == b->grid_fields && b->graph_for_fuse == b->fuse_k)
    return QED_OK;
  drop_graph(b);
  cudaGraph_t g = nullptr;
  const cudaStream_t s = b->own;
  QED_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < b->graph_steps; ++k) launch_batch(b, s);
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  count_launch(-5 * b->graph_steps);  // captured, not executed: replays are counted instead
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { b->graph = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
  b->graph_for_steps = b->graph_steps;
  b->graph_for_target = b->target_blocks;
  b->graph_for_grid = b->grid_fields;
  b->graph_for_fuse = b->fuse_k;
  return QED_OK;
}
}  // namespace

extern "C" qed_status qed_batch_create(const qed_tables* T, qed_precision prec, int S, const qed_allocator* alloc,
                                       void* stream, qed_batch** out) {
  if (!T || !out || S < 1 || S > 4096 || (prec != QED_FP64 && prec != QED_MIXED))
    return fail(QED_ERR_INVALID_ARG, "qed_batch_create: bad argument (1 <= slots <= 4096)");
  *out = nullptr;
  cudaStream_t s = as_stream(stream);
  auto* b = new qed_batch();
  b->tables = T;
  b->precision = prec;
  b->S = S;
  b->target_blocks = step_grid_size(prec);
  if (cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return fail(QED_ERR_CUDA, "qed_batch_create: stream or event creation failed");
  }
  b->max_parts = std::max(step_grid_size(QED_MIXED), step_grid_size(QED_FP64));
  const size_t argb = prec == QED_MIXED ? sizeof(StepArgs<float>) : sizeof(StepArgs<double>);
  Carver cv;
  char* args = nullptr;
  cv.add(&args, argb * S);
  cv.add(&b->remaining, S);
  cv.add(&b->live, S);
  cv.add(&b->blocks, S + 1);
  cv.add(&b->first_event, S);
  cv.add(&b->tried, S);
  cv.add(&b->skip, S);
  cv.add(&b->span, S);
  cv.add(&b->splan, S);
  char* scal = nullptr;
  cv.add(&scal, step_scalars_bytes(prec) * S);
  cv.add(&b->tot, kBatchTotals);
  qed_status st = b->mem.get(cv.total(), alloc, s);
  if (st != QED_OK) { delete b; return st; }
  cv.bind(b->mem.ptr);
  b->args = args;
  b->scal = scal;
  cudaError_t e = cudaMemsetAsync(b->mem.ptr, 0, cv.total(), s);
  if (e != cudaSuccess) { b->mem.release(); delete b; return cuda_fail(e, "cudaMemsetAsync"); }
  *out = b;
  return QED_OK;
}

extern "C" qed_status qed_batch_attach(qed_batch* b, int slot, qed_species* const* sp, const qed_step_params* p,
                                       uint64_t n_steps, void* stream) {
  if (!b || slot < 0 || slot >= b->S) return fail(QED_ERR_INVALID_ARG, "qed_batch_attach: bad slot");
  qed_status st = check_step_args(b->tables, sp, p);
  if (st != QED_OK) return st;
  if (sp[0]->precision != b->precision) return fail(QED_ERR_INVALID_ARG, "qed_batch_attach: precision differs");
  if (n_steps > 0xffffffffull) return fail(QED_ERR_INVALID_ARG, "qed_batch_attach: n_steps must fit 32 bits");
  cudaStream_t s = as_stream(stream);
  st = sync_weights(sp, s);
  if (st != QED_OK) return st;
  const uint32_t rem = (uint32_t)n_steps;
  if (b->precision == QED_MIXED) {
    const StepArgs<float> a = make_args<float>(b->tables, sp, *p, p->step);
    QED_CUDA(cudaMemcpyAsync(static_cast<StepArgs<float>*>(b->args) + slot, &a, sizeof(a), cudaMemcpyHostToDevice, s));
  } else {
    const StepArgs<double> a = make_args<double>(b->tables, sp, *p, p->step);
    QED_CUDA(cudaMemcpyAsync(static_cast<StepArgs<double>*>(b->args) + slot, &a, sizeof(a), cudaMemcpyHostToDevice, s));
  }
  QED_CUDA(cudaMemcpyAsync(b->remaining + slot, &rem, 4, cudaMemcpyHostToDevice, s));
  QED_CUDA(cudaMemsetAsync(b->skip + slot, 0, 4, s));  // a new scenario probes at once,
  QED_CUDA(cudaMemsetAsync(b->span + slot, 0, 4, s));  // over the shortest span first
  QED_CUDA(cudaStreamSynchronize(s));  // the sources are locals
  sp[0]->last_drain = p->drain_photons ? 1 : 0;
  set_slot_grid(b, slot, p->field.kind == QED_FIELD_GRID);
  return QED_OK;
}

extern "C" qed_status qed_batch_detach(qed_batch* b, int slot, void* stream) {
  if (!b || slot < 0 || slot >= b->S) return fail(QED_ERR_INVALID_ARG, "qed_batch_detach: bad slot");
  QED_CUDA(cudaMemsetAsync(b->remaining + slot, 0, 4, as_stream(stream)));
  set_slot_grid(b, slot, false);
  return QED_OK;
}

extern "C" qed_status qed_batch_run(qed_batch* b, uint64_t n_steps, void* stream) {
  if (!b) return fail(QED_ERR_INVALID_ARG, "qed_batch_run: NULL batch");
  cudaStream_t s = as_stream(stream);
  NvtxRange range("qed_batch_run");
  uint64_t done = 0;
  if (b->graph_steps > 0 && n_steps >= (uint64_t)b->graph_steps) {
    qed_status st = ensure_graph(b);
    if (st != QED_OK) return st;
    QED_CUDA(cudaEventRecord(b->ev_in, s));
    QED_CUDA(cudaStreamWaitEvent(b->own, b->ev_in, 0));
    for (; done + b->graph_steps <= n_steps; done += b->graph_steps) {
      QED_CUDA(cudaGraphLaunch(b->graph, b->own));
      count_launch(5 * b->graph_steps);
    }
    QED_CUDA(cudaEventRecord(b->ev_out, b->own));
    QED_CUDA(cudaStreamWaitEvent(s, b->ev_out, 0));
  }
  for (; done < n_steps; ++done) launch_batch(b, s);
  QED_CUDA(cudaGetLastError());
  return QED_OK;
}

extern "C" qed_status qed_batch_remaining(qed_batch* b, uint32_t* out, void* stream) {
  if (!b || !out) return fail(QED_ERR_INVALID_ARG, "qed_batch_remaining: NULL argument");
  QED_CUDA(read_on(out, b->remaining, 4 * (size_t)b->S, as_stream(stream)));
  return QED_OK;
}

extern "C" qed_status qed_batch_config(qed_batch* b, int target_blocks, int graph_steps) {
  if (!b || target_blocks < 0 || target_blocks > b->max_parts || graph_steps < 0 || graph_steps > 4096)
    return fail(QED_ERR_INVALID_ARG, "qed_batch_config: blocks must be in [0, " + std::to_string(b ? b->max_parts : 0) +
                                         "] (one ledger partial each), graph steps in [0, 4096]");
  b->target_blocks = target_blocks > 0 ? target_blocks : step_grid_size(b->precision);
  b->graph_steps = graph_steps;
  return QED_OK;
}

extern "C" qed_status qed_batch_multistep(qed_batch* b, int chunk) {
  if (!b || chunk < 0 || chunk == 1 || chunk > fuse_max_steps())
    return fail(QED_ERR_INVALID_ARG, "qed_batch_multistep: chunk must be 0 or in [2, " +
                                         std::to_string(fuse_max_steps()) + "]");
  b->fuse_k = chunk;
  return QED_OK;
}

extern "C" qed_status qed_batch_tune(qed_batch* b, int trial_steps, int* target_out, int* graph_out, void* stream) {
  if (!b || trial_steps < 1 || !target_out || !graph_out) return fail(QED_ERR_INVALID_ARG, "qed_batch_tune: bad argument");
  cudaStream_t s = as_stream(stream);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = std::max(1, step_grid_size(b->precision) / sms);
  std::vector<std::pair<int, int>> cand;
  for (int bps = 1; bps <= per_sm; ++bps)
    for (int g : {0, 8, 32}) cand.push_back({bps * sms, g});
  cudaEvent_t e0, e1;
  QED_CUDA(cudaEventCreate(&e0));
  QED_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  std::pair<int, int> pick = {b->target_blocks, b->graph_steps};
  // two rounds, so that each candidate is timed at two points of the evolving state
  for (int round = 0; round < 2; ++round)
    for (auto& c : cand) {
      b->target_blocks = c.first;
      b->graph_steps = c.second;
      if (c.second > 0) { qed_status st = ensure_graph(b); if (st != QED_OK) return st; }
      QED_CUDA(cudaEventRecord(e0, s));
      qed_status st = qed_batch_run(b, (uint64_t)std::max(trial_steps, c.second), stream);
      if (st != QED_OK) return st;
      QED_CUDA(cudaEventRecord(e1, s));
      QED_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      QED_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      ms /= (float)std::max(trial_steps, c.second);
      if (round == 1 && ms < best) { best = ms; pick = c; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->target_blocks = pick.first;
  b->graph_steps = pick.second;
  *target_out = pick.first;
  *graph_out = pick.second;
  return QED_OK;
}

extern "C" void qed_batch_free(qed_batch* b) {
  if (!b) return;
  if (b->own) cudaStreamSynchronize(b->own);
  drop_graph(b);
  b->mem.release();
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
}

extern "C" qed_status qed_run(const qed_tables* T, qed_species* const* sp, const qed_step_params* p,
                              uint64_t n_steps, void* stream) {
  qed_status st = check_step_args(T, sp, p);
  if (st != QED_OK) return st;
  cudaStream_t s = as_stream(stream);
  st = sync_weights(sp, s);
  if (st != QED_OK) return st;
  NvtxRange range("qed_run");
  for (uint64_t k = 0; k < n_steps; ++k) {
    st = sp[0]->precision == QED_MIXED ? do_step<float>(T, sp, *p, p->step + k, s)
                                       : do_step<double>(T, sp, *p, p->step + k, s);
    if (st != QED_OK) return st;
  }
  QED_CUDA(cudaGetLastError());
  return QED_OK;
}

extern "C" qed_status qed_step(const qed_tables* T, qed_species* const* sp, const qed_step_params* p, void* stream) {
  return qed_run(T, sp, p, 1, stream);
}

namespace {
// Multi-step runner: probe up to `chunk` steps, commit the event-free stretch in one pass, take
// a step with events on the per-step path.  A probe that finds an event in its first step stops
// early (every thread checks the shared minimum), but still costs a launch and a host
// synchronisation, so after one the runner stays on the per-step path for `chunk` steps.
template <typename R>
qed_status run_multi(const qed_tables* T, qed_species* const* sp, const qed_step_params& p, uint64_t n_steps,
                     int chunk, cudaStream_t s) {
  uint64_t step = p.step, left = n_steps, per_step = 0;
  while (left > 0) {
    if (per_step > 0 || left < 2) {
      const uint64_t m = per_step > 0 ? std::min(left, per_step) : left;
      for (uint64_t k = 0; k < m; ++k) {
        qed_status st = do_step<R>(T, sp, p, step++, s);
        if (st != QED_OK) return st;
      }
      left -= m;
      per_step = 0;
      continue;
    }
    const int K = (int)std::min<uint64_t>((uint64_t)chunk, left);
    StepArgs<R> a = make_args<R>(T, sp, p, step);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool timed = timing_events(e0, e1, g_timing_multi);
    if (timed) cudaEventRecord(e0, s);
    launch_fused<R>(a, K, false, sp[0]->first_event, sp[0]->ledger_parts, s);
    if (timed) cudaEventRecord(e1, s);
    uint32_t k = 0;
    QED_CUDA(cudaMemcpyAsync(&k, sp[0]->first_event, sizeof(k), cudaMemcpyDeviceToHost, s));
    QED_CUDA(cudaStreamSynchronize(s));
    if (k > (uint32_t)K) return fail(QED_ERR_NUMERIC, "qed_run_multistep: bad probe result");
    if (k > 0) {
      a.multi = 1;
      timed = timing_events(e0, e1, g_timing_multi);
      if (timed) cudaEventRecord(e0, s);
      const int grid = launch_fused<R>(a, (int)k, true, sp[0]->first_event, sp[0]->ledger_parts, s);
      if (timed) cudaEventRecord(e1, s);
      launch_finalize<R>(a, grid, s);
      step += k;
      left -= k;
    }
    // step `step` has an event: it goes through the per-step kernels
    if (k < (uint32_t)K) per_step = k == 0 ? (uint64_t)chunk : 1;
  }
  return QED_OK;
}
}  // namespace

extern "C" qed_status qed_run_multistep(const qed_tables* T, qed_species* const* sp, const qed_step_params* p,
                                        uint64_t n_steps, int chunk, void* stream) {
  qed_status st = check_step_args(T, sp, p);
  if (st != QED_OK) return st;
  if (chunk < 2 || chunk > fuse_max_steps())
    return fail(QED_ERR_INVALID_ARG, "qed_run_multistep: chunk must be in [2, " + std::to_string(fuse_max_steps()) + "]");
  cudaStream_t s = as_stream(stream);
  st = sync_weights(sp, s);
  if (st != QED_OK) return st;
  NvtxRange range("qed_run_multistep");
  st = sp[0]->precision == QED_MIXED ? run_multi<float>(T, sp, *p, n_steps, chunk, s)
                                     : run_multi<double>(T, sp, *p, n_steps, chunk, s);
  if (st != QED_OK) return st;
  QED_CUDA(cudaGetLastError());
  return QED_OK;
}

extern "C" qed_status qed_read_ledger(qed_species* const* sp, qed_ledger* out, void* stream) {
  if (!sp || !sp[0] || !out) return fail(QED_ERR_INVALID_ARG, "qed_read_ledger: NULL argument");
  cudaStream_t s = as_stream(stream);
  double v[kLedgerN];
  QED_CUDA(read_on(v, sp[0]->ledger, sizeof(v), s));
  for (int k = 0; k < 3; ++k) { out->n[k] = v[k]; out->energy[k] = v[3 + k]; }
  out->emitted_n = v[6]; out->emitted_energy = v[7]; out->dropped_n = v[8]; out->emit_defect = v[9];
  out->pairs_n = v[10]; out->pair_energy = v[11]; out->pair_defect = v[12];
  out->oor_eta = v[13]; out->oor_chi = v[14];
  out->drained_n = sp[0]->last_drain ? v[6] : 0.0;
  out->drained_energy = sp[0]->last_drain ? v[7] : 0.0;
  return QED_OK;
}

extern "C" qed_status qed_drain_new_particles(qed_species* dr, const qed_soa* dst, size_t cap, size_t* n_out,
                                              void* stream) {
  if (!dr || !dst || !n_out) return fail(QED_ERR_INVALID_ARG, "qed_drain_new_particles: NULL argument");
  cudaStream_t s = as_stream(stream);
  DevCounters c;
  qed_status st = read_counters(dr, c, s);
  if (st != QED_OK) return st;
  if (c.n > cap) return fail(QED_ERR_CAPACITY, "qed_drain_new_particles: destination too small");
  size_t n = 0;
  st = qed_species_download(dr, dst, cap, &n, stream);
  if (st != QED_OK) return st;
  set_counters_kernel<<<1, 1, 0, s>>>(dr->cnt, 0u, c.next_id);
  count_launch();
  QED_CUDA(cudaStreamSynchronize(s));
  *n_out = n;
  return QED_OK;
}

extern "C" qed_status qed_check(qed_species* const* sp, int n_species, void* stream) {
  if (!sp || n_species < 0) return fail(QED_ERR_INVALID_ARG, "qed_check: bad arguments");
  cudaStream_t s = as_stream(stream);
  QED_CUDA(cudaStreamSynchronize(s));
  QED_CUDA(cudaGetLastError());
  qed_status first = QED_OK;
  for (int k = 0; k < n_species; ++k) {
    if (!sp[k]) continue;
    uint32_t err = 0;
    QED_CUDA(read_on(&err, &sp[k]->cnt->err, 4, s));
    if (err) {
      QED_CUDA(cudaMemsetAsync(&sp[k]->cnt->err, 0, 4, s));
      if (first == QED_OK) {
        for (int code = 1; code < 32; ++code)
          if (err & (1u << code)) { first = (qed_status)code; break; }
      }
    }
  }
  if (first != QED_OK) return fail(first, "device reported an error (capacity exceeded or invalid state)");
  return QED_OK;
}

// ============================================================================ diagnostics
extern "C" qed_status qed_eval_particles(const qed_tables* T, qed_precision prec, qed_kind kind,
                                         const qed_field_desc* field, double t, double wx0, double wv, size_t n,
                                         const double* x, const double* y, const double* z, const double* ux,
                                         const double* uy, const double* uz, double* oE, double* oB, double* op,
                                         double* oe, double* orate, void* stream) {
  if (!T || !field || (n && (!x || !y || !z || !ux || !uy || !uz || !oE || !oB || !op || !oe || !orate)))
    return fail(QED_ERR_INVALID_ARG, "qed_eval_particles: NULL argument");
  const qed_status fs = check_field(*field, "qed_eval_particles");
  if (fs != QED_OK) return fs;
  if (n == 0) return QED_OK;
  cudaStream_t s = as_stream(stream);
  const FieldDev f = field_dev(*field);
  if (prec == QED_MIXED) launch_eval<float>(T->d32, f, kind, t, wx0, wv, n, x, y, z, ux, uy, uz, oE, oB, op, oe, orate, s);
  else launch_eval<double>(T->d64, f, kind, t, wx0, wv, n, x, y, z, ux, uy, uz, oE, oB, op, oe, orate, s);
  QED_CUDA(cudaGetLastError());
  return QED_OK;
}

extern "C" qed_status qed_sample(const qed_tables* T, qed_precision prec, int which, size_t n, const double* param,
                                 const double* U, double* out, int32_t* ok, void* stream) {
  if (!T || (n && (!param || !out || !ok || (which < 2 && !U))) || which < 0 || which > 3)
    return fail(QED_ERR_INVALID_ARG, "qed_sample: bad argument");
  if (n == 0) return QED_OK;
  cudaStream_t s = as_stream(stream);
  if (prec == QED_MIXED) launch_sample<float>(T->d32, which, n, param, U, out, ok, s);
  else launch_sample<double>(T->d64, which, n, param, U, out, ok, s);
  QED_CUDA(cudaGetLastError());
  return QED_OK;
}

extern "C" qed_status qed_philox(size_t n, const uint64_t* ctr, const uint64_t key[2], uint64_t* out, void* stream) {
  if (!key || (n && (!ctr || !out))) return fail(QED_ERR_INVALID_ARG, "qed_philox: NULL argument");
  if (n == 0) return QED_OK;
  launch_philox(n, ctr, key[0], key[1], out, as_stream(stream));
  QED_CUDA(cudaGetLastError());
  return QED_OK;
}

extern "C" qed_status qed_work_read(qed_species* e, uint64_t out[3], int reset, void* stream) {
  if (!e || !out) return fail(QED_ERR_INVALID_ARG, "qed_work_read: NULL argument");
  cudaStream_t s = as_stream(stream);
  unsigned long long w[6];
  QED_CUDA(read_on(w, e->work, sizeof(w), s));
  out[0] = w[0];
  out[1] = w[1];
  out[2] = w[2];
  if (reset) QED_CUDA(cudaMemsetAsync(e->work, 0, sizeof(w), s));
  return QED_OK;
}

extern "C" qed_status qed_work_read_split(qed_species* e, uint64_t out[6], int reset, void* stream) {
  if (!e || !out) return fail(QED_ERR_INVALID_ARG, "qed_work_read_split: NULL argument");
  cudaStream_t s = as_stream(stream);
  unsigned long long w[6];
  QED_CUDA(read_on(w, e->work, sizeof(w), s));
  for (int k = 0; k < 6; ++k) out[k] = w[k];
  if (reset) QED_CUDA(cudaMemsetAsync(e->work, 0, sizeof(w), s));
  return QED_OK;
}

extern "C" qed_status qed_timing_enable(int on) {
  g_timing.on = on != 0;
  return QED_OK;
}

extern "C" qed_status qed_timing_read(double* ms, uint64_t* launches, int reset) {
  if (!ms || !launches) return fail(QED_ERR_INVALID_ARG, "qed_timing_read: NULL argument");
  return timing_sum(g_timing, ms, launches, reset);
}

extern "C" qed_status qed_timing_read_multistep(double* ms, uint64_t* passes, int reset) {
  if (!ms || !passes) return fail(QED_ERR_INVALID_ARG, "qed_timing_read_multistep: NULL argument");
  return timing_sum(g_timing_multi, ms, passes, reset);
}

// The self-test's result word: a file-scope device variable, so the self-test allocates nothing.
static __device__ uint32_t g_selftest_bits;

extern "C" qed_status qed_selftest_wait(uint32_t polls, uint32_t* bits_out, void* stream) {
  if (!bits_out || polls == 0) return fail(QED_ERR_INVALID_ARG, "qed_selftest_wait: bad argument");
  cudaStream_t s = as_stream(stream);
  void* d = nullptr;
  QED_CUDA(cudaGetSymbolAddress(&d, g_selftest_bits));
  launch_selftest_wait(polls, static_cast<uint32_t*>(d), s);
  uint32_t h = 0;
  QED_CUDA(read_on(&h, d, sizeof(h), s));
  *bits_out = h;
  return QED_OK;
}

extern "C" uint64_t qed_launch_count(void) { return launch_count_value(); }
extern "C" const char* qed_version(void) { return "qedmc-gb300 0.1 (sm_103a)"; }
extern "C" const char* qed_last_error(void) { return g_err.c_str(); }
