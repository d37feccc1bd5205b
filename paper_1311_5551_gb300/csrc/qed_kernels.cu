// qed_kernels.cu -- CUDA kernels of the QED Monte-Carlo step (Sec. 3) for sm_103a.
//
// One step = one launch of step_kernel over all three species (warp-uniform chunks of 32
// consecutive particles, grid-stride over chunks) followed by three small finalisation
// kernels that merge the particles created during the step in (parent species, parent
// index) order:
//   step_kernel     push, eta/chi, rates, tau; events collected per warp and taken 32 at a time
//                   (ballot + one atomic per warp append), per-chunk event masks, per-block FP64
//                   ledger partials
//   plan_kernel     one block: scans the per-range child counts, checks capacities, writes the
//                   merge plan and reduces the ledger partials in a fixed order
//   prefix_kernel   exclusive prefix of the event-mask popcounts per parent species
//   scatter_kernel  ranks every new particle by its parent's position (a counting sort on the
//                   dense parent index), moves it into place and assigns consecutive ids
#include <cuda_runtime.h>

#include <atomic>

#include "qed_device.cuh"

// The file is compiled three times (QED_KERNELS_PART = 1, 2, 3), so that nvcc builds the
// single-scenario step, the batch step and everything else in parallel: each part defines the
// launchers of its share and so instantiates only their kernels.  Without the macro (0) one
// translation unit holds all of them.
#ifndef QED_KERNELS_PART
#define QED_KERNELS_PART 0
#endif
#define QED_PART(p) (QED_KERNELS_PART == 0 || QED_KERNELS_PART == (p))

namespace qedlib {

namespace {
constexpr unsigned kFull = 0xffffffffu;
constexpr int kBlock = 256;            // compute threads of a step block (one tile of particles)
constexpr int kWarps = kBlock / 32;    // compute warps
constexpr int kStepThreads = kBlock + 32;  // plus one producer warp that issues the tile copies

enum LedgerSlot {
  kN0 = 0, kN1, kN2, kE0, kE1, kE2, kEmitN, kEmitE, kDrop, kEmitDef, kPairN, kPairE, kPairDef, kOorEta, kOorChi,
  kPushedLep, kPushedPh,  // alive particles pushed this step
  kTauPh                  // photons pushed in a field (their optical depth changed and is stored)
};

// Compensated (Kahan) accumulation in the working precision.
template <typename R>
struct KSum {
  R s = (R)0, c = (R)0;  // value = s - c
  __device__ __forceinline__ void add(R v) { const R y = v - c, t = s + y; c = (t - s) - y; s = t; }
  // combine with another compensated sum: exact two-sum of the leading parts, errors folded in
  __device__ __forceinline__ void merge(const KSum& o) {
    const R t = s + o.s;
    const R bb = t - s;
    const R err = (s - (t - bb)) + (o.s - bb);
    c = (c + o.c) - err;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename R>
struct Acc {
  KSum<R> e[3];
  KSum<R> emit_e, emit_def, pair_e, pair_def;
  uint32_t n[3] = {0, 0, 0};
  uint32_t oor_eta = 0, oor_chi = 0;
  uint32_t pushed_lep = 0, pushed_ph = 0, tau_ph = 0;
  uint32_t emit_n = 0, drop = 0, pair_n = 0;
};

// ----------------------------------------------------------------------------- leptons
// Fields at the particle and the Boris push of Sec. 3 (the identity where the field vanishes);
// returns the field case, and what eta_after needs.
template <typename R, bool G, int FC>
struct PushState {
  R E[3], B[3], amp;
};
template <typename R, bool G, int FC>
__device__ __forceinline__ int push_at(const StepScalars<R>& S, R x, R y, R z, R q, R dt, R u[3],
                                       PushState<R, G, FC>& ps) {
  if constexpr (FC == kFieldAny) {
    ps.amp = (R)0;
    const int fc = field_at<R, G>(S, x, y, z, ps.E, ps.B, ps.amp);
    if (fc != kNoField) boris<R>(q, dt, ps.E, ps.B, u);
    return fc;
  } else {
    R ey, ez;
    if (!plane_at<R, FC>(S, x, ey, ez, ps.amp)) return kNoField;
    boris_plane<R, FC>(q, dt, ey, ez, u);
    return kPlaneWave;
  }
}
// eta from u^{n+1/2} in the fields push_at found (Sec. 2; closed form in a plane wave)
template <typename R, bool G, int FC>
__device__ __forceinline__ R eta_after(int fc, const R u[3], R gam, const PushState<R, G, FC>& ps) {
  if constexpr (FC == kFieldAny) return eta_for<R>(fc, u, gam, ps.E, ps.B, ps.amp);
  else return fc == kNoField ? (R)0 : eta_plane<R>(u, gam, ps.amp);
}
// chi of a photon at its position (Sec. 2; closed form in a plane wave), 0 where no field
template <typename R, bool G, int FC>
__device__ __forceinline__ R chi_at(const StepScalars<R>& S, R x, R y, R z, const R k[3], R eps, int& fc) {
  if constexpr (FC == kFieldAny) {
    R E[3], B[3], amp = (R)0;
    fc = field_at<R, G>(S, x, y, z, E, B, amp);
    return chi_for<R>(fc, k, eps, E, B, amp);
  } else {
    R ey, ez, amp;
    if (!plane_at<R, FC>(S, x, ey, ez, amp)) { fc = kNoField; return (R)0; }
    fc = kPlaneWave;
    return chi_plane<R>(k, eps, amp);
  }
}

// The part of a step that every e+- takes (Sec. 3): fields at (x^n, t^n), Boris push to
// u^{n+1/2}, drift to x^{n+1}, eta, and the optical-depth decrement.  Shared by the per-step
// kernel and the multi-step kernels, so both compute the same bits.
template <typename R, bool G, int FC>
__device__ __forceinline__ R lepton_advance(const StepScalars<R>& S, const TabDev<R>& tab, const R* lnh, R q, R dt,
                                            R win_v, R& x, R& y, R& z, R u[3], Tau<R>& tau, R& gam, R& u2, int& oor) {
  using N = Num<R>;
  PushState<R, G, FC> ps;
  // where the field vanishes the push is the identity and eta = 0 (no emission)
  const int fc = push_at<R, G, FC>(S, x, y, z, q, dt, u, ps);
  u2 = dot3<R>(u, u);
  R ig;
  N::root_inv_((R)1 + u2, gam, ig);
  x = N::fma_(dt, N::fma_(u[0], ig, -win_v), x);
  y = N::fma_(dt, u[1] * ig, y);
  z = N::fma_(dt, u[2] * ig, z);
  const R eta = eta_after<R, G, FC>(fc, u, gam, ps);
  oor = 0;
  if (eta > (R)0) {
    const R lam = (R)kRatePhoton * eta * ig * lookup_h<R>(tab, lnh, eta, oor);
    tau.sub(lam * dt);
  }
  return eta;
}

// ----------------------------------------------------------------------------- deferred events
// An event (Sec. 3: a Philox draw, an inverse-CDF search, the recoil or the pair split, the
// appends) is long next to the rest of a particle's step, and rare: a few per warp per step even
// at the peak of a collision.  Taken where it is found, each warp with an event would run that
// path with one lane active.  Instead every warp writes its events into a ring in shared memory
// and takes them 32 at a time, all lanes busy: whenever 32 are waiting, before its next tile is
// of another species, and after its last tile.  An event depends only on its particle's state
// after the push (and its id and weight), so the particles get the same bits as if each event
// were taken where it was found; only the order in which the ledger sums are accumulated changes.
constexpr int kRing = 64;  // entries per warp: fewer than 32 waiting plus at most 32 from a chunk

// The ledger sums that events add to, kept per warp beside its ring (out of the registers of
// the hot loop) and folded into the block's ledger partial at the end.
template <typename R>
struct EventSums {
  KSum<R> e[3], emit_e, emit_def, pair_e, pair_def;
  uint32_t n[3], emit_n, drop, pair_n;
};

template <typename R>
struct __align__(16) EventRing {
  uint32_t i[kRing];  // particle index
  R v[7][kRing];      // x, y, z after the push; u after the push (photons: k); eta (photons: chi)
  EventSums<R> sums;
};

// Compensated warp sum of one value per lane (fixed shuffle order); lane 0 holds the result.
template <typename R>
__device__ __forceinline__ KSum<R> warp_ksum(R v) {
  KSum<R> t;
  t.s = v;
  for (int off = 16; off > 0; off >>= 1) {
    KSum<R> o;
    o.s = __shfl_down_sync(kFull, t.s, off);
    o.c = __shfl_down_sync(kFull, t.c, off);
    t.merge(o);
  }
  return t;
}

// The ring of one warp with its (warp-uniform) head and fill.
template <typename R>
struct EventQueue {
  EventRing<R>* r;
  uint32_t head, count;
};

// Enqueue the warp's events of one chunk (every lane calls this with the chunk's ballot).
template <typename R>
__device__ __forceinline__ void enqueue_event(EventQueue<R>& q, unsigned evm, bool ev, int lane, uint32_t i, R x, R y,
                                              R z, R u0, R u1, R u2, R par) {
  if (ev) {
    const uint32_t p = (q.head + q.count + (uint32_t)__popc(evm & ((1u << lane) - 1u))) & (uint32_t)(kRing - 1);
    q.r->i[p] = i;
    q.r->v[0][p] = x; q.r->v[1][p] = y; q.r->v[2][p] = z;
    q.r->v[3][p] = u0; q.r->v[4][p] = u1; q.r->v[5][p] = u2;
    q.r->v[6][p] = par;
  }
  q.count += (uint32_t)__popc(evm);
}

// One particle of a 32-particle chunk (the whole warp calls this together).  The state comes
// from the shared-memory tile; results are stored straight to global memory.  A particle whose
// optical depth ran out goes to the warp's event ring; its momentum and optical depth are
// stored when the event is taken.  The chunk's event mask counts every event as a child here;
// an emission that yields no photon (below the energy cut) takes its bit back then.
template <typename R, bool G, int FC>
__device__ __forceinline__ void lepton_chunk(const StepArgs<R>& a, const StepScalars<R>& S, const R* lnh, int kind,
                                             uint32_t chunk, uint32_t n, int lane, Acc<R>& acc, EventQueue<R>& q,
                                             R x, R y, R z, R v0, R v1, R v2, const double* tau_src) {
  const SpeciesDev<R>& sp = a.sp[kind];
  const uint32_t i = chunk * 32u + (uint32_t)lane;
  const bool active = i < n;
  R u[3] = {v0, v1, v2};
  Tau<R> tau = Tau<R>::load(tau_src);
  // lanes past the last particle compute on whatever their shared-memory slots hold: nothing
  // they compute is stored, counted or queued, and the table look-ups clamp their indices (a
  // NaN position maps to the first node), so no access leaves its array
  R gam, u2;
  int oor;
  const R eta = lepton_advance<R, G, FC>(S, a.tab, lnh, kind == QED_ELECTRON ? (R)-1 : (R)1, a.dt_r, a.win_v_r, x, y,
                                         z, u, tau, gam, u2, oor);
  if (active && oor > 0) acc.oor_eta++;
  if (active) acc.pushed_lep++;

  const bool ev = active && a.emit && tau.used_up();
  const unsigned evm = __ballot_sync(kFull, ev);
  if (evm) {
    enqueue_event<R>(q, evm, ev, lane, i, x, y, z, u[0], u[1], u[2], eta);
    if (lane == 0) atomicAdd(&sp.rangesum[chunk >> kRangeShift], (uint32_t)__popc(evm));
  }
  if (lane == 0) sp.evmask[chunk] = evm;
  if (active) {
    sp.x[i] = x; sp.y[i] = y; sp.z[i] = z;
    if (!ev) {
      sp.ux[i] = u[0]; sp.uy[i] = u[1]; sp.uz[i] = u[2];
      tau.store(sp.tau + i);
      acc.e[kind].add(gam);
      acc.n[kind]++;
    }
  }
}

// Takes `take` (<= 32) events from the ring, starting at `head`, one per lane: photon emission
// by an e+- (Sec. 3): photon energy from the inverse CDF of P_chi, recoil, fresh optical depths
// for the emitter and the photon, the photon appended to the photon species' append region.
// Inlined into the tile loop: as a call, the ABI's saved registers and the spills around the
// call sites cost the loop more (on GB300, 3 blocks of 288 threads per SM) than the inlined
// code's registers do.
template <typename R, int KIND>
__device__ __forceinline__ void lepton_events(const StepArgs<R>& a, EventRing<R>* ring, uint32_t head, uint32_t take) {
  const SpeciesDev<R>& sp = a.sp[KIND];
  const SpeciesDev<R>& dst = a.sp[2];  // photon children are appended to the photon species
  const int lane = threadIdx.x & 31;
  const bool ev = (uint32_t)lane < take;
  const uint32_t p = (head + (uint32_t)lane) & (uint32_t)(kRing - 1);
  uint32_t i = 0;
  R x = (R)0, y = (R)0, z = (R)0, u[3] = {(R)0, (R)0, (R)0}, eta = (R)0;
  if (ev) {
    i = ring->i[p];
    x = ring->v[0][p]; y = ring->v[1][p]; z = ring->v[2][p];
    u[0] = ring->v[3][p]; u[1] = ring->v[4][p]; u[2] = ring->v[5][p];
    eta = ring->v[6][p];
  }
  // gamma from u after the push, as the push computed it
  const R u2 = dot3<R>(u, u);
  R gam, ig;
  Num<R>::root_inv_((R)1 + u2, gam, ig);
  bool child = false;
  R kx = (R)0, ky = (R)0, kz = (R)0, emitted = (R)0, def = (R)0;
  Tau<R> tau = Tau<R>::one(), ctau = Tau<R>::one();
  if (ev) {
    Uniform<R> U[4];
    draw4r<R>(a.seed, a.scenario, sp.id[i], a.step, (uint64_t)KIND, 0, U);
    R xi;
    if (sample_xi<R>(a.tab, eta, U[0].u, U[0].v, xi)) {
      const R eps = xi * gam;
      const R um = Num<R>::sqrt_(u2);
      const R ium = (R)1 / um;
      const R h0 = u[0] * ium, h1 = u[1] * ium, h2 = u[2] * ium;
      kx = eps * h0; ky = eps * h1; kz = eps * h2;
      // recoil p_f = p_i - (h nu/c) phat_i (Sec. 3), or energy-conserving on request
      R umf;
      if (a.recoil_energy) { const R gf = gam - eps; umf = gf > (R)1 ? Num<R>::sqrt_(gf * gf - (R)1) : (R)0; }
      else umf = um > eps ? um - eps : (R)0;
      u[0] = umf * h0; u[1] = umf * h1; u[2] = umf * h2;
      const R gf = Num<R>::sqrt_((R)1 + umf * umf);
      // energy defect (gamma_f + eps) - gamma_i (Sec. 3.1); for the momentum-conserving recoil
      // written without cancellation as 2 eps / ((gamma_i + |u_i|)(gamma_f + gamma_i - eps))
      if (!a.recoil_energy && um > eps) def = (R)2 * eps / ((gam + um) * (gf + gam - eps));
      else def = (gf + eps) - gam;
      emitted = eps;
      gam = gf;
      ctau = Tau<R>::fresh(-Num<R>::log_(U[2].u));
      child = true;
    } else {
      // no photon: the event is not a child after all
      atomicAnd(&sp.evmask[i >> 5], ~(1u << (i & 31u)));
      atomicSub(&sp.rangesum[(i >> 5) >> kRangeShift], 1u);
    }
    tau = Tau<R>::fresh(-Num<R>::log_(U[1].u));
  }
  const unsigned childm = __ballot_sync(kFull, child);
  const uint32_t nc = (uint32_t)__popc(childm);
  {
    const KSum<R> se = warp_ksum<R>(emitted), sd = warp_ksum<R>(def), sg = warp_ksum<R>(ev ? gam : (R)0);
    if (lane == 0) {
      EventSums<R>& es = ring->sums;
      es.emit_e.merge(se);
      es.emit_def.merge(sd);
      es.emit_n += nc;
      es.drop += take - nc;
      es.e[KIND].merge(sg);
      es.n[KIND] += take;
      if (!a.drain) { es.e[2].merge(se); es.n[2] += nc; }
    }
  }
  if (childm) {
    const int leader = __ffs(childm) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&dst.cnt->n_app, nc);
    base = __shfl_sync(kFull, base, leader);
    if (child) {
      const uint32_t slot = base + (uint32_t)__popc(childm & ((1u << lane) - 1u));
      if (slot < dst.acap) {
        dst.ax[slot] = x; dst.ay[slot] = y; dst.az[slot] = z;
        dst.aux[slot] = kx; dst.auy[slot] = ky; dst.auz[slot] = kz;
        ctau.store(dst.atau + slot);
        dst.aparent[slot] = i | ((uint32_t)KIND << 31);
        if (dst.aw) dst.aw[slot] = sp.w ? sp.w[i] : (R)1;  // the photon stands for as many
      } else {
        atomicOr(&dst.cnt->err, 1u << QED_ERR_CAPACITY);
      }
    }
  }
  if (ev) {
    sp.ux[i] = u[0]; sp.uy[i] = u[1]; sp.uz[i] = u[2];
    tau.store(sp.tau + i);
  }
  __syncwarp();  // the ring slots read above may be refilled by the next chunk
}

// ----------------------------------------------------------------------------- photons
// The part of a step that every photon takes: chi at (x^n, t^n), the pair-rate decrement of the
// optical depth, and the drift at c along k (k does not change between events).
template <typename R, bool G, int FC>
__device__ __forceinline__ R photon_advance(const StepScalars<R>& S, const TabDev<R>& tab, const R* lnT, R dt, R win_v,
                                            R& x, R& y, R& z, const R k[3], Tau<R>& tau, R& eps, R& ie, int& oor) {
  using N = Num<R>;
  N::root_inv_(dot3<R>(k, k), eps, ie);
  int fc;
  const R chi = chi_at<R, G, FC>(S, x, y, z, k, eps, fc);
  oor = 0;
  if (chi > (R)0) {
    const R lam = (R)kAlpha * chi * ie * lookup_T<R>(tab, lnT, chi, oor);
    tau.sub(lam * dt);
  }
  x = N::fma_(dt, N::fma_(k[0], ie, -win_v), x);  // null geodesic at c along khat
  y = N::fma_(dt, k[1] * ie, y);
  z = N::fma_(dt, k[2] * ie, z);
  return chi;
}

template <typename R, bool G, int FC>
__device__ __forceinline__ void photon_chunk(const StepArgs<R>& a, const StepScalars<R>& S, const R* lnT,
                                             uint32_t chunk, uint32_t n, int lane, Acc<R>& acc, EventQueue<R>& q,
                                             R x, R y, R z, R k0, R k1, R k2, const double* tau_src) {
  const SpeciesDev<R>& sp = a.sp[2];
  const uint32_t i = chunk * 32u + (uint32_t)lane;
  Tau<R> tau = Tau<R>::load(tau_src);
  const bool alive = i < n && !tau.dead();  // converted photons stay as holes until compaction
  R k[3] = {k0, k1, k2};
  // dead or past-the-end lanes compute on what their slots hold; none of it is stored (see
  // lepton_chunk)
  R eps, ie;
  int oor;
  const R chi = photon_advance<R, G, FC>(S, a.tab, lnT, a.dt_r, a.win_v_r, x, y, z, k, tau, eps, ie, oor);
  if (alive && oor > 0) acc.oor_chi++;
  if (alive) acc.pushed_ph++;
  // a photon outside any field keeps its optical depth: only its position is stored
  const bool tau_moves = alive && chi > (R)0;
  if (tau_moves) acc.tau_ph++;

  // a photon whose optical depth ran out always converts: its pair is counted here
  const bool ev = alive && a.pairs && tau.used_up();
  const unsigned evm = __ballot_sync(kFull, ev);
  if (evm) {
    enqueue_event<R>(q, evm, ev, lane, i, x, y, z, k[0], k[1], k[2], chi);
    if (lane == 0) {
      const uint32_t c = (uint32_t)__popc(evm);
      atomicAdd(&sp.rangesum[chunk >> kRangeShift], c);
      atomicAdd(&sp.cnt->n_dead, c);
    }
  }
  if (lane == 0) sp.evmask[chunk] = evm;
  if (alive) {
    sp.x[i] = x; sp.y[i] = y; sp.z[i] = z;  // k is unchanged between events
    if (!ev) {
      if (tau_moves) tau.store(sp.tau + i);
      acc.e[2].add(eps);
      acc.n[2]++;
    }
  }
}

// Takes `take` (<= 32) events from the ring, starting at `head`, one per lane: pair creation
// by a photon (Sec. 3): the energy split from the inverse CDF of P_f, the electron and the
// positron along k with fresh optical depths, appended to their species' append regions; the
// photon is annihilated (its optical depth becomes +inf, a hole until compaction).  Inlined
// for the same reason as lepton_events.
template <typename R>
__device__ __forceinline__ void photon_events(const StepArgs<R>& a, EventRing<R>* ring, uint32_t head, uint32_t take) {
  const SpeciesDev<R>& sp = a.sp[2];
  const int lane = threadIdx.x & 31;
  const bool ev = (uint32_t)lane < take;
  const uint32_t p = (head + (uint32_t)lane) & (uint32_t)(kRing - 1);
  uint32_t i = 0;
  R x = (R)0, y = (R)0, z = (R)0, k[3] = {(R)0, (R)0, (R)1}, chi = (R)0;
  if (ev) {
    i = ring->i[p];
    x = ring->v[0][p]; y = ring->v[1][p]; z = ring->v[2][p];
    k[0] = ring->v[3][p]; k[1] = ring->v[4][p]; k[2] = ring->v[5][p];
    chi = ring->v[6][p];
  }
  // the photon energy as the push computed it
  R eps, ie;
  Num<R>::root_inv_(dot3<R>(k, k), eps, ie);
  R ue[3] = {(R)0, (R)0, (R)0}, up[3] = {(R)0, (R)0, (R)0};
  R converted = (R)0, def = (R)0, gm = (R)0, gp = (R)0;
  Tau<R> te = Tau<R>::one(), tp = Tau<R>::one();
  if (ev) {
    Uniform<R> U[4];
    draw4r<R>(a.seed, a.scenario, sp.id[i], a.step, (uint64_t)QED_PHOTON, 0, U);
    const R f = sample_f<R>(a.tab, chi, U[0].u, U[0].v);
    R se = (R)1 - f, sq = f;  // the positron takes f h nu (Sec. 3)
    if (a.recoil_energy && eps >= (R)2) {
      const R g1 = (R)1 + f * (eps - (R)2), g0 = (R)1 + ((R)1 - f) * (eps - (R)2);
      sq = Num<R>::sqrt_(g1 * g1 - (R)1) * ie;
      se = Num<R>::sqrt_(g0 * g0 - (R)1) * ie;
    }
    for (int c = 0; c < 3; ++c) { ue[c] = se * k[c]; up[c] = sq * k[c]; }
    const R pe = se * eps, pp = sq * eps;
    gm = Num<R>::sqrt_((R)1 + pe * pe);
    gp = Num<R>::sqrt_((R)1 + pp * pp);
    // defect (gamma_- + gamma_+) - eps (Sec. 3.1); for the momentum split it is exactly
    // 1/(gamma_- + p_-) + 1/(gamma_+ + p_+), written so to avoid cancellation
    if (!(a.recoil_energy && eps >= (R)2)) def = (R)1 / (gm + pe) + (R)1 / (gp + pp);
    else def = (gm + gp) - eps;
    converted = eps;
    te = Tau<R>::fresh(-Num<R>::log_(U[1].u));
    tp = Tau<R>::fresh(-Num<R>::log_(U[2].u));
  }
  const unsigned evm = __ballot_sync(kFull, ev);
  {
    const KSum<R> se = warp_ksum<R>(converted), sd = warp_ksum<R>(def);
    const KSum<R> s0 = warp_ksum<R>(gm), s1 = warp_ksum<R>(gp);
    if (lane == 0) {
      EventSums<R>& es = ring->sums;
      es.pair_e.merge(se);
      es.pair_def.merge(sd);
      es.pair_n += take;
      es.e[0].merge(s0); es.n[0] += take;
      es.e[1].merge(s1); es.n[1] += take;
    }
  }
  const int leader = __ffs(evm) - 1;
  uint32_t be = 0, bp = 0;
  if (lane == leader) {
    be = atomicAdd(&a.sp[0].cnt->n_app, take);
    bp = atomicAdd(&a.sp[1].cnt->n_app, take);
  }
  be = __shfl_sync(kFull, be, leader);
  bp = __shfl_sync(kFull, bp, leader);
  if (ev) {
    const uint32_t r = (uint32_t)lane;  // the events fill lanes 0 .. take-1
    const SpeciesDev<R>& de = a.sp[0];
    const SpeciesDev<R>& dp = a.sp[1];
    if (be + r < de.acap) {
      const uint32_t s = be + r;
      de.ax[s] = x; de.ay[s] = y; de.az[s] = z;
      de.aux[s] = ue[0]; de.auy[s] = ue[1]; de.auz[s] = ue[2];
      te.store(de.atau + s);
      de.aparent[s] = i;
      if (de.aw) de.aw[s] = sp.w ? sp.w[i] : (R)1;
    } else {
      atomicOr(&de.cnt->err, 1u << QED_ERR_CAPACITY);
    }
    if (bp + r < dp.acap) {
      const uint32_t s = bp + r;
      dp.ax[s] = x; dp.ay[s] = y; dp.az[s] = z;
      dp.aux[s] = up[0]; dp.auy[s] = up[1]; dp.auz[s] = up[2];
      tp.store(dp.atau + s);
      dp.aparent[s] = i;
      if (dp.aw) dp.aw[s] = sp.w ? sp.w[i] : (R)1;
    } else {
      atomicOr(&dp.cnt->err, 1u << QED_ERR_CAPACITY);
    }
    Tau<R>::infinite().store(sp.tau + i);  // the photon is annihilated
  }
  __syncwarp();  // the ring slots read above may be refilled by the next chunk
}

// One pipeline stage: a tile of 256 consecutive particles of one species (8 warp chunks).
constexpr int kTile = kBlock;

template <typename R>
struct TileBuf;

// measured on GB300 at 3 resident blocks per SM (72 registers; 4 blocks per SM spill): on the
// head-on collision of 1e6 electrons 3, 4 and 6 stages tie (2 stages are 7% slower, 8 stages, at
// 2 blocks per SM, 18%); on the 256-scenario scan 4 stages are 16% faster than 6: the shared
// memory they leave to L1 holds the spilled registers and the arguments and tables the event
// paths read
#ifndef QED_STAGES
#define QED_STAGES 4
#endif
#ifndef QED_STEP_MIN_BLOCKS
#define QED_STEP_MIN_BLOCKS 3
#endif
constexpr int kStages = QED_STAGES;  // tile copies in flight per block
constexpr uint32_t kWaitLimit = 1u << 16;  // mbarrier polls (<= 20 us each) before a copy is declared lost

template <typename R>
struct TileBuf {
  R x[kTile], y[kTile], z[kTile], ux[kTile], uy[kTile], uz[kTile];
  double tau[kTile];
};

__device__ __forceinline__ uint32_t floor16(uint32_t b) { return b & ~15u; }

// Tile t of the step (over the concatenated species) -> species and tile index in it.
__device__ __forceinline__ void decode_tile(uint32_t t, uint32_t T0, uint32_t T1, int& s, uint32_t& j) {
  if (t < T0) { s = 0; j = t; }
  else if (t < T0 + T1) { s = 1; j = t - T0; }
  else { s = 2; j = t - T0 - T1; }
}

// Source arrays of species s, selected with constant indices (no dynamic indexing of the
// kernel parameters, which would copy them to local memory).
template <typename R>
struct TileSrc {
  const R *x, *y, *z, *ux, *uy, *uz;
  const double* tau;
};
template <typename R>
__device__ __forceinline__ TileSrc<R> tile_src(const SpeciesDev<R>& p) {
  return {p.x, p.y, p.z, p.ux, p.uy, p.uz, p.tau};
}

// Thread 0 issues the bulk copies of the block's k-th tile into stage k % kStages.
template <typename R>
__device__ __forceinline__ void issue_tile(const StepArgs<R>& a, TileBuf<R>* buf, uint64_t* bar, uint32_t k, uint32_t n0,
                                        uint32_t n1, uint32_t n2, uint32_t blk, uint32_t nblk) {
  const uint32_t T0 = (n0 + kTile - 1) / kTile, T1 = (n1 + kTile - 1) / kTile, T2 = (n2 + kTile - 1) / kTile;
  const uint32_t t = blk + k * nblk;
  if (t >= T0 + T1 + T2) return;
  int s; uint32_t j;
  decode_tile(t, T0, T1, s, j);
  const TileSrc<R> src = s == 0 ? tile_src(a.sp[0]) : (s == 1 ? tile_src(a.sp[1]) : tile_src(a.sp[2]));
  const uint32_t ns = s == 0 ? n0 : (s == 1 ? n1 : n2);
  const uint32_t first = j * kTile;
  const uint32_t valid = min((uint32_t)kTile, ns - first);
  // arrays start 16-byte aligned and tiles start at multiples of 256 particles, so every source
  // is 16-byte aligned; only whole 16-byte pieces are copied (no read past the last particle),
  // the ragged remainder of the last tile is read with plain loads by its threads
  const uint32_t br = floor16(valid * (uint32_t)sizeof(R)), bt = floor16(valid * 8u);
  TileBuf<R>& b = buf[k % kStages];
  uint64_t* bb = &bar[k % kStages];
  mbar_arrive_expect_tx(bb, 6u * br + bt);
  if (br) {
    bulk_load(b.x, src.x + first, br, bb);
    bulk_load(b.y, src.y + first, br, bb);
    bulk_load(b.z, src.z + first, br, bb);
    bulk_load(b.ux, src.ux + first, br, bb);
    bulk_load(b.uy, src.uy + first, br, bb);
    bulk_load(b.uz, src.uz + first, br, bb);
  }
  if (bt) bulk_load(b.tau, src.tau + first, bt, bb);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// barrier among the compute warps only (the producer warp does not take part)
__device__ __forceinline__ void compute_warps_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kBlock) : "memory"); }

// Fixed-order block reduction of the ledger partials in the working precision: compensated
// sums are combined pairwise (two-sum), counts as integers; only the block totals become FP64
// (an FP64 shuffle tree here took a quarter of the kernel on GB300's slow FP64 pipe).
// W warps take part: the whole block (CW = false, every thread calls this), or the compute warps
// only (CW = true, synchronised by their named barrier; the producer warp holds no sums, and its
// zeros would change nothing).
constexpr int kCounts = 11;
template <typename R, int W, bool CW = false>
__device__ __forceinline__ void write_ledger_partial(const Acc<R>& acc, double* ledger_part, uint32_t blk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  KSum<R> f[7] = {acc.e[0], acc.e[1], acc.e[2], acc.emit_e, acc.emit_def, acc.pair_e, acc.pair_def};
  uint32_t c[kCounts] = {acc.n[0], acc.n[1], acc.n[2], acc.emit_n, acc.drop, acc.pair_n, acc.oor_eta, acc.oor_chi,
                         acc.pushed_lep, acc.pushed_ph, acc.tau_ph};
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    KSum<R> t = f[q];
    for (int off = 16; off > 0; off >>= 1) {
      KSum<R> o;
      o.s = __shfl_down_sync(kFull, t.s, off);
      o.c = __shfl_down_sync(kFull, t.c, off);
      t.merge(o);
    }
    f[q] = t;
  }
#pragma unroll
  for (int q = 0; q < kCounts; ++q)
    for (int off = 16; off > 0; off >>= 1) c[q] += __shfl_down_sync(kFull, c[q], off);
  __shared__ KSum<R> s_fr[W][7];
  __shared__ uint32_t s_cr[W][kCounts];
  if (lane == 0) {
    for (int q = 0; q < 7; ++q) s_fr[warp][q] = f[q];
    for (int q = 0; q < kCounts; ++q) s_cr[warp][q] = c[q];
  }
  if (CW) compute_warps_sync();
  else __syncthreads();
  if (threadIdx.x < kLedgerN) {
    const int k = threadIdx.x;
    int fs = -1, cs = -1;  // where ledger field k comes from
    switch (k) {
      case kN0: cs = 0; break;       case kN1: cs = 1; break;       case kN2: cs = 2; break;
      case kE0: fs = 0; break;       case kE1: fs = 1; break;       case kE2: fs = 2; break;
      case kEmitN: cs = 3; break;    case kEmitE: fs = 3; break;    case kDrop: cs = 4; break;
      case kEmitDef: fs = 4; break;  case kPairN: cs = 5; break;    case kPairE: fs = 5; break;
      case kPairDef: fs = 6; break;  case kOorEta: cs = 6; break;   case kOorChi: cs = 7; break;
      case kPushedLep: cs = 8; break; case kPushedPh: cs = 9; break; case kTauPh: cs = 10; break;
      default: break;
    }
    double t = 0.0;
    if (fs >= 0) {
      KSum<R> acc_b = s_fr[0][fs];
      for (int w = 1; w < W; ++w) acc_b.merge(s_fr[w][fs]);
      t = acc_b.value();
    } else if (cs >= 0) {
      uint32_t n = 0;
      for (int w = 0; w < W; ++w) n += s_cr[w][cs];
      t = (double)n;
    }
    ledger_part[(size_t)blk * kLedgerN + k] = t;
  }
  if (CW) compute_warps_sync();  // s_fr and s_cr are reused by the next slot's partial
}

// The block's tiles of species SP, global tiles [t_lo, t_hi), with the block's tile count k
// running on; field class FC.  Events are taken 32 at a time and all of them after the species'
// last tile.  False if a wait gave up (the events left in the ring are then not taken).  One loop
// per species and field class, so no tile decodes its species or dispatches on the field (on
// GB300 this took 10% off the head-on job's per-step kernel).  Species indices stay compile-time
// constants (no dynamic indexing of the kernel parameters, which would copy them to local memory).
template <typename R, bool G, int FC, int SP>
__device__ __forceinline__ bool species_tiles(const StepArgs<R>& a, const StepScalars<R>& S, const R* lnh, const R* lnT,
                                              TileBuf<R>* buf, uint64_t* full, uint64_t* empty, uint32_t& k,
                                              uint32_t blk, uint32_t nblk, uint32_t t_lo, uint32_t t_hi, uint32_t n,
                                              int lane, int warp, Acc<R>& acc, EventQueue<R>& q) {
  const uint32_t last = n ? (n - 1u) / (uint32_t)kTile : 0u;  // the only tile that can be ragged
  const uint32_t valid = n - last * (uint32_t)kTile;
  const uint32_t in_r = floor16(valid * (uint32_t)sizeof(R)) / (uint32_t)sizeof(R);
  const uint32_t in_t = floor16(valid * 8u) / 8u;
  const bool ragged = in_r < valid || in_t < valid;
  const uint32_t r = threadIdx.x;
  for (;; ++k) {
    const uint32_t t = blk + k * nblk;
    const bool more = t < t_hi;
    if (more) {
      const int st = (int)(k % kStages);
      if (!mbar_wait_bounded(&full[st], (k / kStages) & 1u, kWaitLimit)) return false;
      const uint32_t j = t - t_lo;
      TileBuf<R>& b = buf[st];
      if (ragged && j == last) {
        const TileSrc<R> g = tile_src(a.sp[SP]);
        const uint32_t gi = j * kTile + r;
        if (r >= in_r && r < valid) {
          b.x[r] = g.x[gi]; b.y[r] = g.y[gi]; b.z[r] = g.z[gi];
          b.ux[r] = g.ux[gi]; b.uy[r] = g.uy[gi]; b.uz[r] = g.uz[gi];
        }
        if (r >= in_t && r < valid) b.tau[r] = g.tau[gi];
        compute_warps_sync();
      }
      const uint32_t chunk = j * kWarps + warp;
      if (SP == 2)
        photon_chunk<R, G, FC>(a, S, lnT, chunk, n, lane, acc, q, b.x[r], b.y[r], b.z[r], b.ux[r], b.uy[r], b.uz[r],
                               &b.tau[r]);
      else
        lepton_chunk<R, G, FC>(a, S, lnh, SP == 0 ? QED_ELECTRON : QED_POSITRON, chunk, n, lane, acc, q, b.x[r],
                               b.y[r], b.z[r], b.ux[r], b.uy[r], b.uz[r], &b.tau[r]);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
    while (q.count >= 32u || (!more && q.count > 0u)) {
      const uint32_t take = min(q.count, 32u);
      if (SP == 0) lepton_events<R, QED_ELECTRON>(a, q.r, q.head, take);
      else if (SP == 1) lepton_events<R, QED_POSITRON>(a, q.r, q.head, take);
      else photon_events<R>(a, q.r, q.head, take);
      q.head = (q.head + take) & (uint32_t)(kRing - 1);
      q.count -= take;
    }
    if (!more) return true;
  }
}
template <typename R, bool G, int FC>
__device__ __forceinline__ bool species_pass(const StepArgs<R>& a, const StepScalars<R>& S, const R* lnh, const R* lnT,
                                             TileBuf<R>* buf, uint64_t* full, uint64_t* empty, uint32_t& k,
                                             uint32_t blk, uint32_t nblk, uint32_t T0, uint32_t T1, uint32_t ttot,
                                             uint32_t n0, uint32_t n1, uint32_t n2, int lane, int warp, Acc<R>& acc,
                                             EventQueue<R>& q) {
  return species_tiles<R, G, FC, 0>(a, S, lnh, lnT, buf, full, empty, k, blk, nblk, 0u, T0, n0, lane, warp, acc, q) &&
         species_tiles<R, G, FC, 1>(a, S, lnh, lnT, buf, full, empty, k, blk, nblk, T0, T0 + T1, n1, lane, warp, acc,
                                    q) &&
         species_tiles<R, G, FC, 2>(a, S, lnh, lnT, buf, full, empty, k, blk, nblk, T0 + T1, ttot, n2, lane, warp, acc,
                                    q);
}

// The step over one scenario, run by block `blk` of the `nblk` blocks given to it: block blk
// takes the scenario's tiles blk, blk + nblk, ... and writes ledger partial number blk.
// Warp roles: warps 0-7 compute (warp w takes 32-particle chunk w of each tile); warp 8 is the
// producer: its first lane issues the bulk copies of tile k into stage k % kStages once the 8
// compute warps have released that stage (mbarrier `empty`, one arrival per warp); compute warps
// wait only for their tile's data (mbarrier `full`), never for each other.  Each compute warp
// keeps its events in its own ring (see EventRing) and takes them between tiles.
template <typename R, bool G>
__device__ __forceinline__ void step_body(const StepArgs<R>& a, uint32_t blk, uint32_t nblk, unsigned char* smem_raw) {
  TileBuf<R>* buf = reinterpret_cast<TileBuf<R>*>(smem_raw);
  EventRing<R>* ring = reinterpret_cast<EventRing<R>*>(buf + kStages);
  R* s_lnh = reinterpret_cast<R*>(ring + kWarps);
  R* s_lnT = s_lnh + a.tab.n_eta;
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  __shared__ StepScalars<R> S;
  __shared__ int s_abort;

  const uint32_t n0 = a.sp[0].cnt->n, n1 = a.sp[1].cnt->n, n2 = a.sp[2].cnt->n;
  const uint32_t T0 = (n0 + kTile - 1) / kTile, T1 = (n1 + kTile - 1) / kTile, T2 = (n2 + kTile - 1) / kTile;
  const uint32_t ttot = T0 + T1 + T2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kWarps);
    }
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();
  if (threadIdx.x == kBlock)
    for (uint32_t k = 0; k < (uint32_t)kStages; ++k) issue_tile(a, buf, full, k, n0, n1, n2, blk, nblk);
  // stage the rate tables and the per-step field scalars while the first tiles load
  for (int k = threadIdx.x; k < a.tab.n_eta; k += blockDim.x) s_lnh[k] = a.tab.ln_h[k];
  for (int k = threadIdx.x; k < a.tab.n_chi; k += blockDim.x) s_lnT[k] = a.tab.ln_T[k];
  if (threadIdx.x == 0) make_scalars<R>(a.field, a.t0 + (double)a.step * a.dt, a.win_x0, a.win_v, S);
  __syncthreads();

  Acc<R> acc;
  if (warp == kWarps) {
    // ---------------- producer
    if (lane == 0) {
      uint32_t k = kStages;
      for (;; ++k) {
        if (blk + k * nblk >= ttot || s_abort) break;
        const int st = (int)(k % kStages);
        if (!mbar_wait_bounded(&empty[st], ((k / kStages) - 1u) & 1u, kWaitLimit)) { s_abort = 1; break; }
        fence_proxy_async_smem();  // the compute warps' accesses to this stage come first
        issue_tile(a, buf, full, k, n0, n1, n2, blk, nblk);
      }
      if (s_abort) {
        // a wait gave up: report it, then wait (bounded) for the copies this block issued
        atomicOr(&a.sp[0].cnt->err, 1u << QED_ERR_TIMEOUT);
        const uint32_t first = k >= (uint32_t)kStages ? k - kStages : 0u;
        for (uint32_t q = first; q < k; ++q)
          if (blk + q * nblk < ttot) mbar_wait_bounded(&full[q % kStages], (q / kStages) & 1u, kWaitLimit);
      }
    }
  } else {
    // ---------------- compute warps
    EventQueue<R> q{ring + warp, 0u, 0u};
    if (lane == 0) q.r->sums = EventSums<R>{};
    __syncwarp();
    // one loop per species and field class: no per-tile dispatch (a grid-field instantiation
    // only ever sees the general class)
    uint32_t k = 0;
    bool ok;
    if (!G && S.kind == QED_FIELD_PLANE_LP)
      ok = species_pass<R, G, G ? kFieldAny : kFieldLP>(a, S, s_lnh, s_lnT, buf, full, empty, k, blk, nblk, T0, T1,
                                                        ttot, n0, n1, n2, lane, warp, acc, q);
    else if (!G && S.kind == QED_FIELD_PLANE_CP)
      ok = species_pass<R, G, G ? kFieldAny : kFieldCP>(a, S, s_lnh, s_lnT, buf, full, empty, k, blk, nblk, T0, T1,
                                                        ttot, n0, n1, n2, lane, warp, acc, q);
    else
      ok = species_pass<R, G, kFieldAny>(a, S, s_lnh, s_lnT, buf, full, empty, k, blk, nblk, T0, T1, ttot, n0, n1, n2,
                                         lane, warp, acc, q);
    if (!ok) s_abort = 1;
    // a wait that gave up leaves the step unfinished (QED_ERR_TIMEOUT): events still in the
    // ring are not taken
    __syncwarp();
    if (lane == 0) {
      const EventSums<R>& es = q.r->sums;
      for (int c = 0; c < 3; ++c) { acc.e[c].merge(es.e[c]); acc.n[c] += es.n[c]; }
      acc.emit_e = es.emit_e; acc.emit_def = es.emit_def;
      acc.pair_e = es.pair_e; acc.pair_def = es.pair_def;
      acc.emit_n = es.emit_n; acc.drop = es.drop; acc.pair_n = es.pair_n;
    }
  }
  __syncthreads();

  write_ledger_partial<R, kWarps + 1>(acc, a.ledger_part, blk);
}

template <typename R, bool G>
__global__ void __launch_bounds__(kStepThreads, sizeof(R) == 4 ? QED_STEP_MIN_BLOCKS : 1) step_kernel(const StepArgs<R> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  step_body<R, G>(a, blockIdx.x, gridDim.x, smem_raw);
}

// ----------------------------------------------------------------------------- multi-step
// Several steps per pass over the particles, state in registers.  Exact only across steps in
// which no particle has an event (children would have to join and be ordered at their step), so
// it runs in two passes: the probe advances every particle up to K steps without writing
// anything and records the first step (0-based, min over all particles) at which any particle
// would have an event; the commit then advances k <= that many steps and writes the state and
// the ledger of the last of them.  Both run lepton_advance / photon_advance, the per-step
// kernel's own arithmetic, so the particles end up with the bits the per-step kernel gives.
constexpr int kMaxFuse = 64;
constexpr int kFuseThreads = 256;

// State of one particle as the multi-step passes read it (the 7 SoA columns of any species;
// for photons u holds k).
template <typename R>
struct PState {
  R x, y, z, u0, u1, u2;
  double tau;  // stored form
};

// Particle g of the concatenated species (e-, e+, photons): its column pointers.
template <typename R>
struct PCols {
  R *x, *y, *z, *ux, *uy, *uz;
  double* tau;
  uint32_t i;
  int s;
};
template <typename R>
__device__ __forceinline__ PCols<R> cols_of(const StepArgs<R>& a, uint32_t g, uint32_t n0, uint32_t nl) {
  PCols<R> c;
  c.s = g < n0 ? 0 : (g < nl ? 1 : 2);
  c.i = c.s == 0 ? g : (c.s == 1 ? g - n0 : g - nl);
  // constant indices only (no dynamic indexing of the kernel parameters)
  c.x = c.s == 0 ? a.sp[0].x : (c.s == 1 ? a.sp[1].x : a.sp[2].x);
  c.y = c.s == 0 ? a.sp[0].y : (c.s == 1 ? a.sp[1].y : a.sp[2].y);
  c.z = c.s == 0 ? a.sp[0].z : (c.s == 1 ? a.sp[1].z : a.sp[2].z);
  c.ux = c.s == 0 ? a.sp[0].ux : (c.s == 1 ? a.sp[1].ux : a.sp[2].ux);
  c.uy = c.s == 0 ? a.sp[0].uy : (c.s == 1 ? a.sp[1].uy : a.sp[2].uy);
  c.uz = c.s == 0 ? a.sp[0].uz : (c.s == 1 ? a.sp[1].uz : a.sp[2].uz);
  c.tau = c.s == 0 ? a.sp[0].tau : (c.s == 1 ? a.sp[1].tau : a.sp[2].tau);
  return c;
}
template <typename R>
__device__ __forceinline__ PState<R> load_state(const PCols<R>& c) {
  return {c.x[c.i], c.y[c.i], c.z[c.i], c.ux[c.i], c.uy[c.i], c.uz[c.i], c.tau[c.i]};
}

// True when a particle drifting at vx (relative to the window) stays outside a plane-wave
// pulse's envelope through steps 0..K-1 of the stretch: the phase omega (t - x) is linear in the
// step along a straight path, so it suffices that the first and the last step are both on the
// same side of the envelope, with a margin far above the FP32 rounding of the per-step phase
// (the field is then exactly zero at every step, as field_at would find).
template <typename R>
__device__ __forceinline__ bool outside_pulse(const StepScalars<R>* S, int K, R x, R vx, R dt) {
  if (S[0].kind != QED_FIELD_PLANE_LP && S[0].kind != QED_FIELD_PLANE_CP) return false;
  if (!(S[0].len > (R)0)) return false;
  using N = Num<R>;
  const R ph0 = N::fma_(-S[0].omega, x, S[0].phi_ref);
  const R ph1 = N::fma_(-S[0].omega, N::fma_((R)(K - 1) * dt, vx, x), S[K - 1].phi_ref);
  const R m0 = (R)1e-2 + (R)1e-5 * fabs(ph0), m1 = (R)1e-2 + (R)1e-5 * fabs(ph1);
  return (ph0 < -m0 && ph1 < -m1) || (ph0 > S[0].len + m0 && ph1 > S[0].len + m1);
}

// One scenario's multi-step pass, run by block `blk` of the `nblk` blocks given to it (all
// threads of the block call it).
template <typename R, bool G, bool COMMIT, int FC>
__device__ __forceinline__ void fused_body(const StepArgs<R>& a, int K, uint32_t* first_event, uint32_t blk,
                                           uint32_t nblk, unsigned char* smem_raw) {
  R* s_lnh = reinterpret_cast<R*>(smem_raw);
  R* s_lnT = s_lnh + a.tab.n_eta;
  __shared__ StepScalars<R> S[kMaxFuse];
  for (int k = threadIdx.x; k < a.tab.n_eta; k += blockDim.x) s_lnh[k] = a.tab.ln_h[k];
  for (int k = threadIdx.x; k < a.tab.n_chi; k += blockDim.x) s_lnT[k] = a.tab.ln_T[k];
  if ((int)threadIdx.x < K)
    make_scalars<R>(a.field, a.t0 + (double)(a.step + threadIdx.x) * a.dt, a.win_x0, a.win_v, S[threadIdx.x]);
  __syncthreads();

  const uint32_t n0 = a.sp[0].cnt->n, n1 = a.sp[1].cnt->n, n2 = a.sp[2].cnt->n;
  const uint32_t nl = n0 + n1, tot = nl + n2;
  const uint32_t stride = nblk * blockDim.x;
  const R dt = a.dt_r, wv = a.win_v_r;
  using N = Num<R>;
  Acc<R> acc;
  bool bad = false;
  uint32_t g = blk * blockDim.x + threadIdx.x;
  // the next particle's state is loaded while the current one is stepped
  PCols<R> cc = cols_of(a, g < tot ? g : 0u, n0, nl);
  PState<R> cur;
  if (g < tot) cur = load_state(cc);
  for (; g < tot; g += stride) {
    const uint32_t gn = g + stride;
    const PCols<R> nc = cols_of(a, gn < tot ? gn : g, n0, nl);
    PState<R> nxt;
    if (gn < tot) nxt = load_state(nc);
    int limit = K;
    if (!COMMIT) {
      // no need to simulate past the earliest event found so far
      limit = min(K, (int)*reinterpret_cast<volatile uint32_t*>(first_event));
      if (limit == 0) break;
    }
    R x = cur.x, y = cur.y, z = cur.z;
    Tau<R> tau = Tau<R>::from_stored(cur.tau);
    int k = 0;
    if (cc.s < 2) {
      const bool pos = cc.s == 1;
      R u[3] = {cur.u0, cur.u1, cur.u2};
      const R q = pos ? (R)1 : (R)-1;
      // lepton_advance, step by step, with the drift velocity kept while u does not change
      // (where the field vanishes the push is the identity): the same operations on the same
      // values, so the same bits
      R gam, ig;
      N::root_inv_((R)1 + dot3<R>(u, u), gam, ig);
      R vx = N::fma_(u[0], ig, -wv), vy = u[1] * ig, vz = u[2] * ig;
      int oor = 0;
      if (outside_pulse<R>(S, limit, x, vx, dt)) {
        // no field at any step of the stretch: the drift only (nothing to probe)
        if (COMMIT)
          for (; k < limit; ++k) { x = N::fma_(dt, vx, x); y = N::fma_(dt, vy, y); z = N::fma_(dt, vz, z); }
        else
          k = limit;
      }
      for (; k < limit; ++k) {
        PushState<R, G, FC> ps;
        const int fc = push_at<R, G, FC>(S[k], x, y, z, q, dt, u, ps);
        if (fc == kNoField) {
          x = N::fma_(dt, vx, x); y = N::fma_(dt, vy, y); z = N::fma_(dt, vz, z);
          oor = 0;
          continue;  // no rate, no event
        }
        N::root_inv_((R)1 + dot3<R>(u, u), gam, ig);
        vx = N::fma_(u[0], ig, -wv); vy = u[1] * ig; vz = u[2] * ig;
        x = N::fma_(dt, vx, x); y = N::fma_(dt, vy, y); z = N::fma_(dt, vz, z);
        const R eta = eta_after<R, G, FC>(fc, u, gam, ps);
        oor = 0;
        if (eta > (R)0) {
          const R lam = (R)kRatePhoton * eta * ig * lookup_h<R>(a.tab, s_lnh, eta, oor);
          tau.sub(lam * dt);
        }
        if (a.emit && tau.used_up()) break;
      }
      if (!COMMIT) {
        if (k < limit) atomicMin(first_event, (uint32_t)k);
      } else {
        bad |= k < K;  // the probe ruled this out; the arithmetic is the same
        cc.x[cc.i] = x; cc.y[cc.i] = y; cc.z[cc.i] = z;
        cc.ux[cc.i] = u[0]; cc.uy[cc.i] = u[1]; cc.uz[cc.i] = u[2];
        tau.store(cc.tau + cc.i);
        acc.e[pos ? 1 : 0].add(gam);
        acc.n[pos ? 1 : 0]++;
        acc.pushed_lep += (uint32_t)K;
        if (oor > 0) acc.oor_eta++;
      }
    } else if (!tau.dead()) {  // converted photons stay as holes until compaction
      const R kv[3] = {cur.u0, cur.u1, cur.u2};
      // photon_advance, step by step: k does not change, so neither do eps, 1/eps and the drift
      R eps, ie;
      N::root_inv_(dot3<R>(kv, kv), eps, ie);
      const R vx = N::fma_(kv[0], ie, -wv), vy = kv[1] * ie, vz = kv[2] * ie;
      int oor = 0;
      if (outside_pulse<R>(S, limit, x, vx, dt)) {
        if (COMMIT)
          for (; k < limit; ++k) { x = N::fma_(dt, vx, x); y = N::fma_(dt, vy, y); z = N::fma_(dt, vz, z); }
        else
          k = limit;
      }
      for (; k < limit; ++k) {
        int fc;
        const R chi = chi_at<R, G, FC>(S[k], x, y, z, kv, eps, fc);
        oor = 0;
        if (fc != kNoField) {
          if (chi > (R)0) {
            const R lam = (R)kAlpha * chi * ie * lookup_T<R>(a.tab, s_lnT, chi, oor);
            tau.sub(lam * dt);
          }
        }
        x = N::fma_(dt, vx, x); y = N::fma_(dt, vy, y); z = N::fma_(dt, vz, z);
        if (fc != kNoField && a.pairs && tau.used_up()) break;
      }
      if (!COMMIT) {
        if (k < limit) atomicMin(first_event, (uint32_t)k);
      } else {
        bad |= k < K;
        cc.x[cc.i] = x; cc.y[cc.i] = y; cc.z[cc.i] = z;
        tau.store(cc.tau + cc.i);
        acc.e[2].add(eps);
        acc.n[2]++;
        acc.pushed_ph += (uint32_t)K;
        if (oor > 0) acc.oor_chi++;
      }
    }
    cc = nc;
    cur = nxt;
  }
  if (COMMIT) {
    if (bad) atomicOr(&a.sp[0].cnt->err, 1u << QED_ERR_NUMERIC);
    __syncthreads();
    write_ledger_partial<R, kFuseThreads / 32>(acc, a.ledger_part, blk);
  }
}

template <typename R, bool G, bool COMMIT>
__global__ void __launch_bounds__(kFuseThreads) fused_kernel(const StepArgs<R> a, int K, uint32_t* first_event) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // the field class of the run (every step of a stretch has the same field)
  if (a.field.kind == QED_FIELD_PLANE_LP)
    fused_body<R, G, COMMIT, kFieldLP>(a, K, first_event, blockIdx.x, gridDim.x, smem_raw);
  else if (a.field.kind == QED_FIELD_PLANE_CP)
    fused_body<R, G, COMMIT, kFieldCP>(a, K, first_event, blockIdx.x, gridDim.x, smem_raw);
  else
    fused_body<R, G, COMMIT, kFieldAny>(a, K, first_event, blockIdx.x, gridDim.x, smem_raw);
}

__global__ void set_u32_kernel(uint32_t* p, uint32_t v) { *p = v; }

// Failure-detection self-test of the bounded mbarrier wait that every pipeline wait uses: a
// barrier whose phase completes is waited for successfully; a barrier that nothing ever arrives
// at gives up after `polls` polls instead of hanging.  bits: 1 = completed wait returned true,
// 2 = unsatisfiable wait timed out.
__global__ void selftest_wait_kernel(uint32_t polls, uint32_t* bits) {
  __shared__ __align__(8) uint64_t done_bar, never_bar;
  if (threadIdx.x == 0) {
    mbar_init(&done_bar, 1);
    mbar_init(&never_bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t out = 0;
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&done_bar)) : "memory");
    if (mbar_wait_bounded(&done_bar, 0u, polls)) out |= 1u;
    if (!mbar_wait_bounded(&never_bar, 0u, polls)) out |= 2u;
    *bits = out;
  }
}


// ----------------------------------------------------------------------------- finalisation
// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024, multiple of 32).
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t s_w[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  uint32_t inc = v;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, inc, off);
    if (lane >= off) inc += t;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nwarp ? s_w[lane] : 0u;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, w, off);
      if (lane >= off) w += t;
    }
    s_w[lane] = w;  // inclusive prefix over warps
  }
  __syncthreads();
  const uint32_t warp_base = warp > 0 ? s_w[warp - 1] : 0u;
  if (total) *total = s_w[nwarp - 1];
  __syncthreads();
  return warp_base + inc - v;
}

template <typename R>
__device__ __forceinline__ void plan_body(const StepArgs<R>& a, int nparts) {
  __shared__ uint32_t s_tot[3];
  constexpr int kPer = 8;  // range sums a thread keeps in registers (more go through memory twice)
  for (int s = 0; s < 3; ++s) {
    const SpeciesDev<R>& sp = a.sp[s];
    const uint32_t words = (sp.cnt->n + 31u) >> 5;
    const uint32_t ranges = (words + (1u << kRangeShift) - 1u) >> kRangeShift;
    // each thread scans a contiguous segment of ranges; the loads of a segment are issued
    // together and kept for the write-back
    const uint32_t per = (ranges + blockDim.x - 1) / blockDim.x;
    const uint32_t r0 = threadIdx.x * per, r1 = min(ranges, r0 + per);
    uint32_t v[kPer];
    uint32_t local = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      v[q] = (q < (int)per && r0 + q < r1) ? sp.rangesum[r0 + q] : 0u;
      local += v[q];
    }
    for (uint32_t r = r0 + kPer; r < r1; ++r) local += sp.rangesum[r];
    uint32_t total;
    uint32_t run = block_exclusive_scan(local, &total);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      if (q < (int)per && r0 + q < r1) {
        sp.rprefix[r0 + q] = run;
        run += v[q];
        sp.rangesum[r0 + q] = 0u;  // ready for the next step
      }
    }
    for (uint32_t r = r0 + kPer; r < r1; ++r) {
      const uint32_t c = sp.rangesum[r];
      sp.rprefix[r] = run;
      run += c;
      sp.rangesum[r] = 0u;
    }
    if (threadIdx.x == 0) {
      s_tot[s] = total;
      a.plan->ranges[s] = ranges;
      a.plan->events[s] = total;
    }
  }
  __syncthreads();
  // destinations e-, e+, photons checked by threads 0, 1, 2 at once
  if (threadIdx.x < 3) {
    const int d = threadIdx.x;
    FinalizePlan& P = *a.plan;
    const uint32_t pairs = a.pairs ? s_tot[2] : 0u;
    const uint32_t photons = a.emit ? s_tot[0] + s_tot[1] : 0u;
    const SpeciesDev<R>& dst = (d == 2 && a.drain) ? a.sp[3] : (d == 0 ? a.sp[0] : (d == 1 ? a.sp[1] : a.sp[2]));
    const SpeciesDev<R>& app = d == 0 ? a.sp[0] : (d == 1 ? a.sp[1] : a.sp[2]);  // append region owner
    const uint32_t n_old = dst.cnt->n, next_old = dst.cnt->next_id, n_app = app.cnt->n_app;
    P.n_old[d] = n_old;
    P.next_id_old[d] = next_old;
    uint32_t m = d == 2 ? photons : pairs;
    if (n_app != m || m > app.acap) {  // an append overflowed: drop the step's children
      atomicOr(&dst.cnt->err, 1u << QED_ERR_CAPACITY);
      m = 0;
    }
    if ((uint64_t)n_old + m > dst.cap) {
      atomicOr(&dst.cnt->err, 1u << QED_ERR_CAPACITY);
      m = 0;
    }
    P.m[d] = m;
    if (d == 0) P.from_electrons = s_tot[0];
  }
  // ledger: fixed-order reduction of the per-block partials, one warp per ledger field (lane l
  // sums partials l, l+32, ... in order, then a fixed shuffle tree): deterministic for a fixed grid
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < kLedgerN; k += blockDim.x >> 5) {
    double t = 0.0;
#pragma unroll 4
    for (int p = lane; p < nparts; p += 32) t += a.ledger_part[(size_t)p * kLedgerN + k];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(kFull, t, off);
    if (lane == 0) {
      a.ledger[k] = t;
      // several warps update the work counters: integer atomics (order-independent)
      if (k == kPushedLep) atomicAdd(&a.work[0], (unsigned long long)t);
      if (!a.multi && k == kTauPh) atomicAdd(&a.work[5], (unsigned long long)t);
      if (k == kPushedPh) atomicAdd(&a.work[1], (unsigned long long)t);
      if (a.multi && k == kPushedLep) atomicAdd(&a.work[3], (unsigned long long)t);
      if (a.multi && k == kPushedPh) atomicAdd(&a.work[4], (unsigned long long)t);
      if (k == kEmitN) atomicAdd(&a.work[2], (unsigned long long)t);
      if (k == kPairN) atomicAdd(&a.work[2], 2ull * (unsigned long long)t);
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(1024) plan_kernel(const StepArgs<R> a, int nparts) {
  plan_body<R>(a, nparts);
}

template <typename R>
__device__ __forceinline__ void prefix_body(const StepArgs<R>& a, uint32_t bx, uint32_t gx) {
  const uint32_t R0 = a.plan->ranges[0], R1 = a.plan->ranges[1], R2 = a.plan->ranges[2];
  for (uint32_t g = bx; g < R0 + R1 + R2; g += gx) {
    const int s = g < R0 ? 0 : (g < R0 + R1 ? 1 : 2);
    const uint32_t r = g - (s == 0 ? 0u : (s == 1 ? R0 : R0 + R1));
    const SpeciesDev<R>& sp = a.sp[s];
    // ranges without events hold no parent of any child: their word prefixes are never read
    // (the test is uniform across the block, as the scan below needs)
    const uint32_t Rs = s == 0 ? R0 : (s == 1 ? R1 : R2);
    const uint32_t r_end = r + 1 < Rs ? sp.rprefix[r + 1] : a.plan->events[s];
    if (r_end == sp.rprefix[r]) continue;
    const uint32_t words = (sp.cnt->n + 31u) >> 5;
    const uint32_t w = (r << kRangeShift) + threadIdx.x;
    const uint32_t m = w < words ? sp.evmask[w] : 0u;
    const uint32_t ex = block_exclusive_scan((uint32_t)__popc(m), nullptr);
    if (w < words) sp.wprefix[w] = sp.rprefix[r] + ex;
  }
}

template <typename R>
__global__ void __launch_bounds__(256) prefix_kernel(const StepArgs<R> a) {
  prefix_body<R>(a, blockIdx.x, gridDim.x);
}

template <typename R>
__device__ __forceinline__ uint32_t parent_rank(const SpeciesDev<R>& ps, uint32_t p) {
  const uint32_t w = p >> 5, b = p & 31u;
  return ps.wprefix[w] + (uint32_t)__popc(ps.evmask[w] & ((1u << b) - 1u));
}

// Child c (in destination order e-, e+, photons) of the step planned in P: its rank among the
// destination's new particles is its parent's rank (a counting sort on the dense parent index),
// which fixes its slot and its id.
template <typename R>
__device__ __forceinline__ void scatter_one(const StepArgs<R>& a, const FinalizePlan& P, uint32_t c) {
  const uint32_t m0 = P.m[0], m1 = P.m[1];
  const int d = c < m0 ? 0 : (c < m0 + m1 ? 1 : 2);
  const uint32_t j = c - (d == 0 ? 0u : (d == 1 ? m0 : m0 + m1));
  const SpeciesDev<R>& app = a.sp[d];
  const SpeciesDev<R>& dst = (d == 2 && a.drain) ? a.sp[3] : a.sp[d];
  const uint32_t par = app.aparent[j];
  uint32_t rank;
  if (d < 2) {
    rank = parent_rank(a.sp[2], par);
  } else {
    const uint32_t pk = par >> 31;
    rank = parent_rank(a.sp[pk], par & 0x7fffffffu) + (pk ? P.from_electrons : 0u);
  }
  if (rank >= P.m[d]) { atomicOr(&dst.cnt->err, 1u << QED_ERR_NUMERIC); return; }
  const uint32_t o = P.n_old[d] + rank;
  dst.x[o] = app.ax[j]; dst.y[o] = app.ay[j]; dst.z[o] = app.az[j];
  dst.ux[o] = app.aux[j]; dst.uy[o] = app.auy[j]; dst.uz[o] = app.auz[j];
  dst.tau[o] = app.atau[j];
  dst.id[o] = P.next_id_old[d] + rank;
  if (dst.w) dst.w[o] = app.aw ? app.aw[j] : (R)1;
}

// The counters after the merge (one thread).
template <typename R>
__device__ __forceinline__ void finish_counters(const StepArgs<R>& a, const FinalizePlan& P) {
  for (int d = 0; d < 3; ++d) {
    const SpeciesDev<R>& dst = (d == 2 && a.drain) ? a.sp[3] : a.sp[d];
    dst.cnt->n = P.n_old[d] + P.m[d];
    dst.cnt->next_id = P.next_id_old[d] + P.m[d];
    a.sp[d].cnt->n_app = 0u;
  }
}

template <typename R>
__device__ __forceinline__ void scatter_body(const StepArgs<R>& a, uint32_t bx, uint32_t gx) {
  const FinalizePlan P = *a.plan;
  const uint32_t tot = P.m[0] + P.m[1] + P.m[2];
  for (uint32_t c = bx * blockDim.x + threadIdx.x; c < tot; c += gx * blockDim.x) scatter_one<R>(a, P, c);
  if (bx == 0 && threadIdx.x == 0) finish_counters<R>(a, P);
}

template <typename R>
__global__ void __launch_bounds__(256) scatter_kernel(const StepArgs<R> a) {
  scatter_body<R>(a, blockIdx.x, gridDim.x);
}

// ----------------------------------------------------------------------------- batches
// Copies one slot's arguments into shared memory (8-byte words, all threads).
template <typename R>
__device__ __forceinline__ void load_args(StepArgs<R>& dst, const StepArgs<R>* src) {
  static_assert(sizeof(StepArgs<R>) % 8 == 0, "StepArgs is a whole number of 8-byte words");
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(StepArgs<R>) / 8); k += blockDim.x) d[k] = s[k];
  __syncthreads();
}

// One block: which slots step now and how many step-kernel blocks each gets (proportional to
// its 256-particle tiles, at least one for a slot with work, at most its ledger partials).
template <typename R>
__global__ void __launch_bounds__(1024) batch_schedule_kernel(const BatchCtl<R> c) {
  __shared__ unsigned long long s_tiles;
  if (threadIdx.x == 0) s_tiles = 0ull;
  __syncthreads();
  const int per = (c.S + blockDim.x - 1) / blockDim.x;
  unsigned long long mine = 0;
  for (int q = 0; q < per; ++q) {
    const int sl = threadIdx.x * per + q;
    if (sl >= c.S || c.remaining[sl] == 0u) continue;
    const StepArgs<R>& a = c.args[sl];
    for (int k = 0; k < 3; ++k) mine += (a.sp[k].cnt->n + kTile - 1) / kTile;
  }
  atomicAdd(&s_tiles, mine);
  __syncthreads();
  const double total = (double)s_tiles;
  uint32_t local = 0;
  for (int q = 0; q < per; ++q) {
    const int sl = threadIdx.x * per + q;
    if (sl >= c.S) continue;
    uint32_t b = 0;
    const bool live = c.remaining[sl] > 0u;
    if (live) {
      const StepArgs<R>& a = c.args[sl];
      uint32_t t = 0;
      for (int k = 0; k < 3; ++k) t += (a.sp[k].cnt->n + kTile - 1) / kTile;
      if (t > 0) {
        b = (uint32_t)(c.target_blocks * (double)t / total + 0.5);
        b = max(1u, min(b, min(t, (uint32_t)c.max_parts)));
      }
    }
    c.live[sl] = live ? 1u : 0u;
    local += b;
  }
  uint32_t tot;
  uint32_t run = block_exclusive_scan(local, &tot);
  for (int q = 0; q < per; ++q) {
    const int sl = threadIdx.x * per + q;
    if (sl >= c.S) continue;
    c.blocks[sl] = run;
    if (c.live[sl]) {
      const StepArgs<R>& a = c.args[sl];
      uint32_t t = 0;
      for (int k = 0; k < 3; ++k) t += (a.sp[k].cnt->n + kTile - 1) / kTile;
      if (t > 0) {
        uint32_t b = (uint32_t)(c.target_blocks * (double)t / total + 0.5);
        run += max(1u, min(b, min(t, (uint32_t)c.max_parts)));
      }
    }
  }
  if (threadIdx.x == blockDim.x - 1) c.blocks[c.S] = tot;
}

// Slot of block b: the last slot whose first block is <= b (blocks[] is non-decreasing).
__device__ __forceinline__ int slot_of_block(const uint32_t* blocks, int S, uint32_t b) {
  int lo = 0, hi = S;  // blocks[lo] <= b < blocks[hi]
  while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (blocks[mid] <= b) lo = mid; else hi = mid; }
  return lo;
}

// ---- per-step path of a batch: one tile space over all live slots
// The tile schedule (one block) lays the live slots' tiles end to end (slot order, species order
// inside a slot), and likewise their event-mask ranges, and evaluates every slot's per-step field
// scalars once.
template <typename R>
__global__ void __launch_bounds__(1024) batch_tiles_kernel(const BatchCtl<R> c) {
  const int per = (c.S + blockDim.x - 1) / blockDim.x;
  const int s0 = threadIdx.x * per, s1 = min(c.S, s0 + per);
  uint32_t tiles = 0, ranges = 0;
  for (int sl = s0; sl < s1; ++sl) {
    SlotPlan q{};
    q.live = c.remaining[sl] > 0u ? 1u : 0u;
    if (q.live) {
      const StepArgs<R>& a = c.args[sl];
      for (int k = 0; k < 3; ++k) {
        q.n[k] = a.sp[k].cnt->n;
        q.T[k] = (q.n[k] + kTile - 1) / kTile;
        const uint32_t words = (q.n[k] + 31u) >> 5;
        q.Rg[k] = (words + (1u << kRangeShift) - 1u) >> kRangeShift;
        tiles += q.T[k];
        ranges += q.Rg[k];
      }
      make_scalars<R>(a.field, a.t0 + (double)a.step * a.dt, a.win_x0, a.win_v,
                      static_cast<StepScalars<R>*>(c.scal)[sl]);
    }
    c.splan[sl] = q;
  }
  uint32_t ttot, rtot;
  uint32_t tb = block_exclusive_scan(tiles, &ttot);
  uint32_t rb = block_exclusive_scan(ranges, &rtot);
  for (int sl = s0; sl < s1; ++sl) {
    SlotPlan& q = c.splan[sl];
    q.tile_base = tb;
    q.range_base = rb;
    tb += q.T[0] + q.T[1] + q.T[2];
    rb += q.Rg[0] + q.Rg[1] + q.Rg[2];
    c.live[sl] = q.live;
  }
  if (threadIdx.x == 0) { c.tot[0] = ttot; c.tot[1] = rtot; }
}

// The run of tiles of one (slot, species) that global tile g of the batch step lies in: its tiles
// are [g_lo, g_hi) of the tile space, slot_lo the slot's first.  A block's tiles increase, so the
// slot cursor only moves forward and the run is looked up again only when g leaves it.
struct TileRun {
  int slot = 0, s = -1;
  uint32_t g_lo = 0, g_hi = 0, slot_lo = 0;
  uint32_t n = 0;  // particles of the species (the step's parents)
};
__device__ __forceinline__ void find_run(const SlotPlan* sp, int S, uint32_t g, TileRun& r) {
  if (g >= r.g_lo && g < r.g_hi) return;
  int cur = r.slot;
  while (cur + 1 < S && sp[cur + 1].tile_base <= g) ++cur;
  const SlotPlan& q = sp[cur];
  const uint32_t local = g - q.tile_base, T0 = q.T[0], T1 = q.T[1];
  r.slot = cur;
  r.slot_lo = q.tile_base;
  if (local < T0) { r.s = 0; r.g_lo = q.tile_base; r.g_hi = r.g_lo + T0; r.n = q.n[0]; }
  else if (local < T0 + T1) { r.s = 1; r.g_lo = q.tile_base + T0; r.g_hi = r.g_lo + T1; r.n = q.n[1]; }
  else { r.s = 2; r.g_lo = q.tile_base + T0 + T1; r.g_hi = r.g_lo + q.T[2]; r.n = q.n[2]; }
}

// Producer (thread kBlock): bulk copies of the block's k-th tile, global tile g, into stage
// k % kStages; as issue_tile, with the arrays of the tile's run (kept while the run lasts).
template <typename R>
__device__ __forceinline__ void issue_batch_tile(const BatchCtl<R>& c, TileBuf<R>* buf, uint64_t* bar, uint32_t k,
                                                 uint32_t g, TileRun& run, TileSrc<R>& src) {
  if (!(g >= run.g_lo && g < run.g_hi)) {
    find_run(c.splan, c.S, g, run);
    src = tile_src(c.args[run.slot].sp[run.s]);
  }
  const TileSrc<R>& sp = src;
  const uint32_t first = (g - run.g_lo) * kTile;
  const uint32_t valid = min((uint32_t)kTile, run.n - first);
  const uint32_t br = floor16(valid * (uint32_t)sizeof(R)), bt = floor16(valid * 8u);
  TileBuf<R>& b = buf[k % kStages];
  uint64_t* bb = &bar[k % kStages];
  mbar_arrive_expect_tx(bb, 6u * br + bt);
  if (br) {
    bulk_load(b.x, sp.x + first, br, bb);
    bulk_load(b.y, sp.y + first, br, bb);
    bulk_load(b.z, sp.z + first, br, bb);
    bulk_load(b.ux, sp.ux + first, br, bb);
    bulk_load(b.uy, sp.uy + first, br, bb);
    bulk_load(b.uz, sp.uz + first, br, bb);
  }
  if (bt) bulk_load(b.tau, sp.tau + first, bt, bb);
}

// The block's tiles of one run (slot, species SP: global tiles [run.g_lo, run.g_hi)), the block's
// tile count k running on; field class FC.  Events are taken 32 at a time and all of them after
// the run's last tile.  Once a wait gave up (`stopped`) the tiles are passed over.
template <typename R, bool G, int FC, int SP>
__device__ __forceinline__ void run_tiles(const StepArgs<R>& A, const StepScalars<R>& S, const R* lnh, const R* lnT,
                                          TileBuf<R>* buf, uint64_t* full, uint64_t* empty, uint32_t& k, uint32_t blk,
                                          uint32_t nblk, const TileRun& run, int lane, int warp, Acc<R>& acc,
                                          EventQueue<R>& q, bool& stopped, int& s_abort) {
  const uint32_t n = run.n;
  const uint32_t last = n ? (n - 1u) / (uint32_t)kTile : 0u;  // the only tile that can be ragged
  const uint32_t valid = n - last * (uint32_t)kTile;
  const uint32_t in_r = floor16(valid * (uint32_t)sizeof(R)) / (uint32_t)sizeof(R);
  const uint32_t in_t = floor16(valid * 8u) / 8u;
  const bool ragged = in_r < valid || in_t < valid;
  const uint32_t r = threadIdx.x;
  for (;; ++k) {
    const uint32_t g = blk + k * nblk;
    const bool more = g < run.g_hi;
    if (more) {
      const int st = (int)(k % kStages);
      if (!stopped && (s_abort || !mbar_wait_bounded(&full[st], (k / kStages) & 1u, kWaitLimit))) {
        s_abort = 1;
        stopped = true;
      }
      if (stopped) continue;
      TileBuf<R>& b = buf[st];
      const uint32_t j = g - run.g_lo;
      // the ragged remainder of a species' last tile: each thread reads its own particle
      if (ragged && j == last && r < valid && (r >= in_r || r >= in_t)) {
        const SpeciesDev<R>& gs = A.sp[SP];
        const uint32_t gi = j * kTile + r;
        if (r >= in_r) {
          b.x[r] = gs.x[gi]; b.y[r] = gs.y[gi]; b.z[r] = gs.z[gi];
          b.ux[r] = gs.ux[gi]; b.uy[r] = gs.uy[gi]; b.uz[r] = gs.uz[gi];
        }
        if (r >= in_t) b.tau[r] = gs.tau[gi];
      }
      const uint32_t chunk = j * kWarps + warp;
      if (SP == 2)
        photon_chunk<R, G, FC>(A, S, lnT, chunk, n, lane, acc, q, b.x[r], b.y[r], b.z[r], b.ux[r], b.uy[r], b.uz[r],
                               &b.tau[r]);
      else
        lepton_chunk<R, G, FC>(A, S, lnh, SP == 0 ? QED_ELECTRON : QED_POSITRON, chunk, n, lane, acc, q, b.x[r],
                               b.y[r], b.z[r], b.ux[r], b.uy[r], b.uz[r], &b.tau[r]);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
    if (stopped) {
      if (!more) return;
      continue;
    }
    while (q.count >= 32u || (!more && q.count > 0u)) {
      const uint32_t take = min(q.count, 32u);
      if (SP == 0) lepton_events<R, QED_ELECTRON>(A, q.r, q.head, take);
      else if (SP == 1) lepton_events<R, QED_POSITRON>(A, q.r, q.head, take);
      else photon_events<R>(A, q.r, q.head, take);
      q.head = (q.head + take) & (uint32_t)(kRing - 1);
      q.count -= take;
    }
    if (!more) return;
  }
}
template <typename R, bool G, int FC>
__device__ __forceinline__ void run_species(const StepArgs<R>& A, const StepScalars<R>& S, const R* lnh, const R* lnT,
                                            TileBuf<R>* buf, uint64_t* full, uint64_t* empty, uint32_t& k,
                                            uint32_t blk, uint32_t nblk, const TileRun& run, int lane, int warp,
                                            Acc<R>& acc, EventQueue<R>& q, bool& stopped, int& s_abort) {
  if (run.s == 0)
    run_tiles<R, G, FC, 0>(A, S, lnh, lnT, buf, full, empty, k, blk, nblk, run, lane, warp, acc, q, stopped, s_abort);
  else if (run.s == 1)
    run_tiles<R, G, FC, 1>(A, S, lnh, lnT, buf, full, empty, k, blk, nblk, run, lane, warp, acc, q, stopped, s_abort);
  else
    run_tiles<R, G, FC, 2>(A, S, lnh, lnT, buf, full, empty, k, blk, nblk, run, lane, warp, acc, q, stopped, s_abort);
}

// One batch step of every live slot in one persistent launch.  Block blk takes the global tiles
// blk, blk + G, blk + 2G, ... (G = gridDim.x), whatever slot they belong to, so every block gets
// an equal share of tiles in one wave.  Inside a slot, block blk takes exactly the slot-local
// tiles j = p, p + G, ... (p: its first one) that block p takes when the slot runs alone with the
// same grid, and writes ledger partial p: a scenario's ledger partials, and so its ledger, are the
// same alone and in any mix.  The warp roles, the pipeline and the per-warp event rings are those
// of step_body; the compute warps switch to a slot's arguments and field scalars together (named
// barrier) when their tiles move on to the next slot, after taking the events queued for it and
// writing its ledger partial.
template <typename R, bool G>
__global__ void __launch_bounds__(kStepThreads, sizeof(R) == 4 ? QED_STEP_MIN_BLOCKS : 1)
batch_step_kernel(const BatchCtl<R> c) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TileBuf<R>* buf = reinterpret_cast<TileBuf<R>*>(smem_raw);
  EventRing<R>* ring = reinterpret_cast<EventRing<R>*>(buf + kStages);
  R* s_lnh = reinterpret_cast<R*>(ring + kWarps);
  R* s_lnT = s_lnh + c.tab.n_eta;
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  __shared__ __align__(16) StepArgs<R> A;
  __shared__ __align__(16) StepScalars<R> S;
  __shared__ int s_abort;

  const uint32_t blk = blockIdx.x, nblk = gridDim.x;
  const uint32_t ttot = c.tot[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kWarps);
    }
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();
  TileRun prun;  // producer's run of tiles and its arrays
  TileSrc<R> psrc{};
  if (threadIdx.x == kBlock)
    for (uint32_t k = 0; k < (uint32_t)kStages && blk + k * nblk < ttot; ++k)
      issue_batch_tile(c, buf, full, k, blk + k * nblk, prun, psrc);
  for (int k = threadIdx.x; k < c.tab.n_eta; k += blockDim.x) s_lnh[k] = c.tab.ln_h[k];
  for (int k = threadIdx.x; k < c.tab.n_chi; k += blockDim.x) s_lnT[k] = c.tab.ln_T[k];
  __syncthreads();

  if (warp == kWarps) {
    // ---------------- producer
    if (lane == 0) {
      uint32_t k = kStages;
      for (;; ++k) {
        if (blk + k * nblk >= ttot || s_abort) break;
        const int st = (int)(k % kStages);
        if (!mbar_wait_bounded(&empty[st], ((k / kStages) - 1u) & 1u, kWaitLimit)) { s_abort = 1; break; }
        fence_proxy_async_smem();
        issue_batch_tile(c, buf, full, k, blk + k * nblk, prun, psrc);
      }
      if (s_abort) {
        atomicOr(&c.args[0].sp[0].cnt->err, 1u << QED_ERR_TIMEOUT);
        const uint32_t first = k >= (uint32_t)kStages ? k - kStages : 0u;
        for (uint32_t q = first; q < k; ++q)
          if (blk + q * nblk < ttot) mbar_wait_bounded(&full[q % kStages], (q / kStages) & 1u, kWaitLimit);
      }
    }
    return;  // the producer takes part in no later barrier
  }
  // ---------------- compute warps
  EventQueue<R> q{ring + warp, 0u, 0u};
  Acc<R> acc;
  if (lane == 0) q.r->sums = EventSums<R>{};
  __syncwarp();
  TileRun run;
  int cur = -1;
  uint32_t part = 0;
  bool stopped = false;  // a wait gave up: no more waits or work, but every slot barrier is kept
  const int nw = (int)(sizeof(StepArgs<R>) / 8), ns = (int)(sizeof(StepScalars<R>) / 8);
  static_assert(sizeof(StepArgs<R>) % 8 == 0 && sizeof(StepScalars<R>) % 8 == 0, "8-byte words");
  auto flush_slot = [&]() {
    __syncwarp();
    if (lane == 0) {
      const EventSums<R>& es = q.r->sums;
      for (int k = 0; k < 3; ++k) { acc.e[k].merge(es.e[k]); acc.n[k] += es.n[k]; }
      acc.emit_e = es.emit_e; acc.emit_def = es.emit_def;
      acc.pair_e = es.pair_e; acc.pair_def = es.pair_def;
      acc.emit_n = es.emit_n; acc.drop = es.drop; acc.pair_n = es.pair_n;
      q.r->sums = EventSums<R>{};
    }
    __syncwarp();
    write_ledger_partial<R, kWarps, true>(acc, A.ledger_part, part);
    acc = Acc<R>{};
  };
  for (uint32_t k = 0;;) {
    const uint32_t g = blk + k * nblk;
    if (g >= ttot) break;
    find_run(c.splan, c.S, g, run);
    if (run.slot != cur) {
      if (cur >= 0) flush_slot();
      compute_warps_sync();  // every warp is done with the previous slot's arguments
      const unsigned long long* sa = reinterpret_cast<const unsigned long long*>(c.args + run.slot);
      const unsigned long long* ss = reinterpret_cast<const unsigned long long*>(
          static_cast<const StepScalars<R>*>(c.scal) + run.slot);
      unsigned long long* da = reinterpret_cast<unsigned long long*>(&A);
      unsigned long long* ds = reinterpret_cast<unsigned long long*>(&S);
      for (int w = threadIdx.x; w < nw; w += kBlock) da[w] = sa[w];
      for (int w = threadIdx.x; w < ns; w += kBlock) ds[w] = ss[w];
      compute_warps_sync();
      cur = run.slot;
      part = g - run.slot_lo;  // < G: the block's first tile of the slot
    }
    // the block's tiles of this run (one slot, one species), compiled for its species and field
    // class (a batch with a grid field runs the grid-capable instantiation: the general class only)
    if (!G && S.kind == QED_FIELD_PLANE_LP)
      run_species<R, G, G ? kFieldAny : kFieldLP>(A, S, s_lnh, s_lnT, buf, full, empty, k, blk, nblk, run, lane, warp,
                                                  acc, q, stopped, s_abort);
    else if (!G && S.kind == QED_FIELD_PLANE_CP)
      run_species<R, G, G ? kFieldAny : kFieldCP>(A, S, s_lnh, s_lnT, buf, full, empty, k, blk, nblk, run, lane, warp,
                                                  acc, q, stopped, s_abort);
    else
      run_species<R, G, kFieldAny>(A, S, s_lnh, s_lnT, buf, full, empty, k, blk, nblk, run, lane, warp, acc, q, stopped,
                                   s_abort);
  }
  // a wait that gave up leaves the step unfinished (QED_ERR_TIMEOUT): events still in the ring
  // are not taken
  if (cur >= 0) flush_slot();
}

// Per-slot plan (one block per live slot): as plan_kernel, over the slot's partials
// 0 .. min(its tiles, G) - 1.
template <typename R>
__global__ void __launch_bounds__(1024) batch_plan_kernel(const BatchCtl<R> c, int G) {
  __shared__ __align__(16) StepArgs<R> A;
  const int sl = blockIdx.x;
  const SlotPlan& q = c.splan[sl];
  if (!q.live) return;
  const uint32_t tiles = q.T[0] + q.T[1] + q.T[2];
  load_args(A, c.args + sl);
  plan_body<R>(A, (int)min(tiles, (uint32_t)G));
}

// Event-mask prefixes of every live slot's ranges with events, one warp per range over the
// batch step's range space (ranges without events are never read by the scatter).
template <typename R>
__global__ void __launch_bounds__(256) batch_prefix_kernel(const BatchCtl<R> c) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const uint32_t rtot = c.tot[1];
  int cur = 0;
  for (uint32_t rg = gw; rg < rtot; rg += nw) {
    while (cur + 1 < c.S && c.splan[cur + 1].range_base <= rg) ++cur;
    const SlotPlan& q = c.splan[cur];
    uint32_t r = rg - q.range_base;
    int s = 0;
    if (r >= q.Rg[0]) { r -= q.Rg[0]; s = 1; if (r >= q.Rg[1]) { r -= q.Rg[1]; s = 2; } }
    const StepArgs<R>& a = c.args[cur];
    const SpeciesDev<R>& sp = a.sp[s];
    const uint32_t r0 = sp.rprefix[r];
    const uint32_t r_end = r + 1 < q.Rg[s] ? sp.rprefix[r + 1] : a.plan->events[s];
    if (r_end == r0) continue;
    const uint32_t words = (q.n[s] + 31u) >> 5;
    const uint32_t w0 = (r << kRangeShift) + lane * 8u;
    uint32_t pc[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      pc[i] = w0 + i < words ? (uint32_t)__popc(sp.evmask[w0 + i]) : 0u;
      sum += pc[i];
    }
    uint32_t inc = sum;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, inc, off);
      if (lane >= (uint32_t)off) inc += t;
    }
    uint32_t run = r0 + inc - sum;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (w0 + i < words) sp.wprefix[w0 + i] = run;
      run += pc[i];
    }
  }
}

// The new particles of every live slot, ranked and moved into place (scatter_one) by a grid that
// strides through all slots' children together; the first threads of block 0 then set each
// slot's counters and advance its step.
constexpr int kMaxScatterSlots = 4096;
template <typename R>
__global__ void __launch_bounds__(256) batch_scatter_kernel(const BatchCtl<R> c) {
  __shared__ uint32_t s_base[kMaxScatterSlots + 1];
  const int per = (c.S + blockDim.x - 1) / blockDim.x;
  const int s0 = threadIdx.x * per, s1 = min(c.S, s0 + per);
  uint32_t mine = 0;
  for (int sl = s0; sl < s1; ++sl) {
    uint32_t m = 0;
    if (c.splan[sl].live) { const FinalizePlan* P = c.args[sl].plan; m = P->m[0] + P->m[1] + P->m[2]; }
    s_base[sl] = m;
    mine += m;
  }
  __syncthreads();
  uint32_t tot;
  uint32_t run = block_exclusive_scan(mine, &tot);
  for (int sl = s0; sl < s1; ++sl) { const uint32_t m = s_base[sl]; s_base[sl] = run; run += m; }
  if (threadIdx.x == 0) s_base[c.S] = tot;
  __syncthreads();
  for (uint32_t ci = blockIdx.x * blockDim.x + threadIdx.x; ci < tot; ci += gridDim.x * blockDim.x) {
    int lo = 0, hi = c.S;  // s_base[lo] <= ci < s_base[hi]
    while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (s_base[mid] <= ci) lo = mid; else hi = mid; }
    const StepArgs<R>& a = c.args[lo];
    scatter_one<R>(a, *a.plan, ci - s_base[lo]);
  }
  if (blockIdx.x == 0)
    for (int sl = threadIdx.x; sl < c.S; sl += blockDim.x) {
      if (!c.splan[sl].live) continue;
      const StepArgs<R>& a = c.args[sl];
      finish_counters<R>(a, *a.plan);
      c.args[sl].step = a.step + 1;  // the slot's next step
      c.remaining[sl] -= 1u;
    }
}

// Multi-step passes in a batch (when fuse_k >= 2): every live slot probes up to
// min(fuse_k, remaining) steps, commits its event-free stretch and advances by it; then the
// regular batch step follows, so a batch step moves a slot by one step plus its stretch.  Each
// slot runs the single-scenario bodies, so its particles are those of qed_run.
// A probe costs a pass over the slot's particles for up to its span of steps, so the span
// adapts per slot: it doubles (up to fuse_k) after a probe that found no event, shrinks to what
// was found otherwise, and a probe that finds an event in the first step makes the slot wait
// fuse_k batch steps before probing again.
template <typename R>
__global__ void __launch_bounds__(1024) batch_probe_init_kernel(const BatchCtl<R> c) {
  for (int sl = threadIdx.x; sl < c.S; sl += blockDim.x) {
    uint32_t k = 0;
    if (c.live[sl]) {
      if (c.skip[sl] > 0) c.skip[sl] -= 1u;
      else k = min(max(c.span[sl], 2u), min((uint32_t)c.fuse_k, c.remaining[sl]));
    }
    c.first_event[sl] = k;
    c.tried[sl] = k;
  }
}

template <typename R, bool G, bool COMMIT>
__global__ void __launch_bounds__(kFuseThreads) batch_fused_kernel(const BatchCtl<R> c) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(16) StepArgs<R> A;
  __shared__ int s_K;
  const uint32_t b = blockIdx.x;
  if (b >= c.blocks[c.S]) return;
  const int sl = slot_of_block(c.blocks, c.S, b);
  // probe: the stretch still worth trying (other blocks of the slot may be lowering it right
  // now); commit: the event-free steps the probe found.  Read once, so that the whole block
  // takes the same branch and copies the arguments together.
  if (threadIdx.x == 0) s_K = (int)*reinterpret_cast<volatile uint32_t*>(c.first_event + sl);
  __syncthreads();
  const int K = s_K;
  if (K == 0) return;
  load_args(A, c.args + sl);
  const uint32_t bb = b - c.blocks[sl], nb = c.blocks[sl + 1] - c.blocks[sl];
  if (A.field.kind == QED_FIELD_PLANE_LP) fused_body<R, G, COMMIT, kFieldLP>(A, K, c.first_event + sl, bb, nb, smem_raw);
  else if (A.field.kind == QED_FIELD_PLANE_CP) fused_body<R, G, COMMIT, kFieldCP>(A, K, c.first_event + sl, bb, nb, smem_raw);
  else fused_body<R, G, COMMIT, kFieldAny>(A, K, c.first_event + sl, bb, nb, smem_raw);
}

template <typename R>
__global__ void __launch_bounds__(1024) batch_commit_plan_kernel(const BatchCtl<R> c) {
  __shared__ __align__(16) StepArgs<R> A;
  const int sl = blockIdx.x;
  const uint32_t k = c.first_event[sl], tried = c.tried[sl];
  if (threadIdx.x == 0 && tried > 0) {
    if (k == 0) c.skip[sl] = (uint32_t)c.fuse_k;
    c.span[sl] = k == tried ? min(2u * tried, (uint32_t)c.fuse_k) : max(k, 2u);
  }
  if (k == 0) return;
  load_args(A, c.args + sl);
  if (threadIdx.x == 0) A.multi = 1;
  __syncthreads();
  plan_body<R>(A, (int)(c.blocks[sl + 1] - c.blocks[sl]));  // no children: counters stay, ledger of the last step
  __syncthreads();
  if (threadIdx.x == 0) {
    c.args[sl].step = A.step + k;
    c.remaining[sl] -= k;
  }
}

// ----------------------------------------------------------------------------- utilities
template <typename R>
__global__ void init_tau_kernel(const SpeciesDev<R> sp, int kind, uint64_t seed, uint64_t scen) {
  const uint32_t n = sp.cnt->n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double U[4];
    draw4(seed, scen, sp.id[i], 0, (uint64_t)kind, 1, U);
    store_tau_from_double<R>(sp.tau + i, -log(U[0]));
  }
}

template <typename R>
__global__ void eval_kernel(const TabDev<R> tab, const FieldDev f, int kind, double t, double wx0, double wv, size_t n,
                            const double* x, const double* y, const double* z, const double* ux, const double* uy,
                            const double* uz, double* oE, double* oB, double* op, double* oe, double* orate) {
  __shared__ StepScalars<R> S;
  if (threadIdx.x == 0) make_scalars<R>(f, t, wx0, wv, S);
  __syncthreads();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    R E[3], B[3], amp = (R)0, u[3] = {(R)ux[i], (R)uy[i], (R)uz[i]};
    const int fc = field_at<R, true>(S, (R)x[i], (R)y[i], (R)z[i], E, B, amp);
    int oor;
    R param, energy, inv, rate;
    // the step's own forms: energy and its inverse from one reciprocal square root, the
    // quantum parameter for the field case, the same look-ups
    if (kind == QED_PHOTON) {
      Num<R>::root_inv_(dot3<R>(u, u), energy, inv);
      param = chi_for<R>(fc, u, energy, E, B, amp);
      rate = param > (R)0 ? (R)kAlpha * param * inv * lookup_T<R>(tab, tab.ln_T, param, oor) : (R)0;
    } else {
      Num<R>::root_inv_((R)1 + dot3<R>(u, u), energy, inv);
      param = eta_for<R>(fc, u, energy, E, B, amp);
      rate = param > (R)0 ? (R)kRatePhoton * param * inv * lookup_h<R>(tab, tab.ln_h, param, oor) : (R)0;
    }
    for (int c = 0; c < 3; ++c) { oE[3 * i + c] = (double)E[c]; oB[3 * i + c] = (double)B[c]; }
    op[i] = (double)param;
    oe[i] = (double)energy;
    orate[i] = (double)rate;
  }
}

template <typename R>
__global__ void sample_kernel(const TabDev<R> tab, int which, size_t n, const double* param, const double* U,
                              double* out, int32_t* ok) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (which >= 2) {
      // the step's rate look-ups for a given parameter, from the tables staged as the step does
      int oor = 0;
      const R v = which == 2 ? lookup_h<R>(tab, tab.ln_h, (R)param[i], oor) : lookup_T<R>(tab, tab.ln_T, (R)param[i], oor);
      out[i] = (double)v;
      ok[i] = oor;
      continue;
    }
    const R u = (R)U[i], v = (R)(1.0 - U[i]);
    if (which == 0) {
      R xi = (R)0;
      const bool good = sample_xi<R>(tab, (R)param[i], u, v, xi);
      out[i] = good ? (double)xi : 0.0;
      ok[i] = good ? 1 : 0;
    } else {
      out[i] = (double)sample_f<R>(tab, (R)param[i], u, v);
      ok[i] = 1;
    }
  }
}

__global__ void philox_kernel(size_t n, const uint64_t* ctr, uint64_t k0, uint64_t k1, uint64_t* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint64_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    philox4x64(c, k0, k1);
    for (int j = 0; j < 4; ++j) out[4 * i + j] = c[j];
  }
}

// ----------------------------------------------------------------------------- tau format
// In-place conversion between the C ABI's double optical depth and the stored representation
// (identical for FP64; a compensated float pair for the mixed path).  Exact round trip.
template <typename R>
__global__ void tau_from_double_kernel(double* tau, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    store_tau_from_double<R>(tau + i, tau[i]);
}
template <typename R>
__global__ void tau_to_double_kernel(double* tau, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    tau[i] = tau_to_double<R>(tau + i);
}

// ----------------------------------------------------------------------------- compaction
// Stable removal of converted photons (tau = +inf) into a second array set, three passes over
// segments of 2048 particles: count survivors, scan the counts (one block), scatter in order.
constexpr uint32_t kSeg = 2048;

template <typename R>
__global__ void __launch_bounds__(256) compact_count_kernel(const SpeciesDev<R> sp, uint32_t* seg_count) {
  const uint32_t n = sp.cnt->n, nseg = (n + kSeg - 1) / kSeg;
  for (uint32_t g = blockIdx.x; g < nseg; g += gridDim.x) {
    uint32_t c = 0;
    for (uint32_t i = g * kSeg + threadIdx.x; i < min(n, (g + 1) * kSeg); i += blockDim.x)
      c += !Tau<R>::load(sp.tau + i).dead();
    uint32_t tot;
    block_exclusive_scan(c, &tot);
    if (threadIdx.x == 0) seg_count[g] = tot;
  }
}

template <typename R>
__global__ void __launch_bounds__(1024) compact_scan_kernel(const SpeciesDev<R> sp, uint32_t* seg_count,
                                                             uint32_t* seg_prefix) {
  const uint32_t n = sp.cnt->n, nseg = (n + kSeg - 1) / kSeg;
  const uint32_t per = (nseg + blockDim.x - 1) / blockDim.x;
  const uint32_t r0 = threadIdx.x * per, r1 = min(nseg, r0 + per);
  uint32_t local = 0;
  for (uint32_t r = r0; r < r1; ++r) local += seg_count[r];
  uint32_t total;
  uint32_t run = block_exclusive_scan(local, &total);
  for (uint32_t r = r0; r < r1; ++r) { seg_prefix[r] = run; run += seg_count[r]; }
  if (threadIdx.x == 0) seg_prefix[nseg] = total;
}

template <typename R>
__global__ void __launch_bounds__(256) compact_scatter_kernel(const SpeciesDev<R> sp, SpeciesDev<R> out,
                                                              const uint32_t* seg_prefix) {
  const uint32_t n = sp.cnt->n, nseg = (n + kSeg - 1) / kSeg;
  for (uint32_t g = blockIdx.x; g < nseg; g += gridDim.x) {
    uint32_t base = seg_prefix[g];
    for (uint32_t i0 = g * kSeg; i0 < min(n, (g + 1) * kSeg); i0 += blockDim.x) {
      const uint32_t i = i0 + threadIdx.x;
      const bool keep = i < n && !Tau<R>::load(sp.tau + i).dead();
      uint32_t tot;
      const uint32_t ex = block_exclusive_scan(keep ? 1u : 0u, &tot);
      if (keep) {
        const uint32_t o = base + ex;
        out.x[o] = sp.x[i]; out.y[o] = sp.y[i]; out.z[o] = sp.z[i];
        out.ux[o] = sp.ux[i]; out.uy[o] = sp.uy[i]; out.uz[o] = sp.uz[i];
        out.tau[o] = sp.tau[i]; out.id[o] = sp.id[i];
        if (sp.w) out.w[o] = sp.w[i];
      }
      base += tot;
    }
  }
}

// The new count, once every block of the scatter has read the old one.
template <typename R>
__global__ void compact_finish_kernel(const SpeciesDev<R> sp, const uint32_t* seg_prefix) {
  const uint32_t n = sp.cnt->n, nseg = (n + kSeg - 1) / kSeg;
  sp.cnt->n = seg_prefix[nseg];
  sp.cnt->n_dead = 0;
}

std::atomic<uint64_t> g_launches{0};
int g_sm_count = 0;

int sm_count() {
  if (g_sm_count == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    g_sm_count = v > 0 ? v : 1;
  }
  return g_sm_count;
}

int small_grid(size_t n) {
  const size_t want = (n + 255) / 256;
  const size_t cap = (size_t)sm_count() * 8;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}
}  // namespace

#if QED_PART(1)
void count_launch(int n) { g_launches += (uint64_t)n; }
uint64_t launch_count_value() { return g_launches.load(); }
#endif

// dynamic shared memory of the step kernel: the tile stages, the compute warps' event rings,
// then ln h and ln T
template <typename R>
static size_t step_smem(int n_eta, int n_chi) {
  return (size_t)kStages * sizeof(TileBuf<R>) + (size_t)kWarps * sizeof(EventRing<R>) +
         (size_t)(n_eta + n_chi) * sizeof(R);
}

template <typename R>
static int step_blocks_per_sm(size_t smem) {
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(step_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, step_kernel<R, false>, kStepThreads, smem);
  return b > 0 ? b : 1;
}

#if QED_PART(1)
int step_grid_size(int precision) {
  // occupancy for the paper's table sizes (256 eta, 256 chi)
  const int b = precision == QED_MIXED ? step_blocks_per_sm<float>(step_smem<float>(256, 256))
                                       : step_blocks_per_sm<double>(step_smem<double>(256, 256));
  return sm_count() * b;
}

template <typename R>
void launch_step(const StepArgs<R>& a, int grid, int block, size_t smem_unused, cudaStream_t s) {
  (void)block;
  (void)smem_unused;
  const size_t smem = step_smem<R>(a.tab.n_eta, a.tab.n_chi);
  // the grid-capable instantiation runs in waves if it fits fewer blocks per SM; the analytic-field
  // one sets the persistent grid size
  if (a.field.kind == QED_FIELD_GRID) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(step_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    step_kernel<R, true><<<grid, kStepThreads, smem, s>>>(a);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(step_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    step_kernel<R, false><<<grid, kStepThreads, smem, s>>>(a);
  }
  count_launch();
}

#endif

#if QED_PART(2)
template <typename R>
void launch_batch_step(const BatchCtl<R>& c, int n_eta, int n_chi, cudaStream_t s) {
  const size_t smem = step_smem<R>(n_eta, n_chi);
  if (smem + sizeof(StepArgs<R>) + sizeof(StepScalars<R>) > 40 * 1024) {
    cudaFuncSetAttribute(batch_step_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(batch_step_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (c.fuse_k >= 2) {
    const size_t fsm = (size_t)(n_eta + n_chi) * sizeof(R);
    const int fgrid = c.target_blocks + c.S;
    batch_schedule_kernel<R><<<1, 1024, 0, s>>>(c);
    batch_probe_init_kernel<R><<<1, 1024, 0, s>>>(c);
    if (c.grid_fields) {
      batch_fused_kernel<R, true, false><<<fgrid, kFuseThreads, fsm, s>>>(c);
      batch_fused_kernel<R, true, true><<<fgrid, kFuseThreads, fsm, s>>>(c);
    } else {
      batch_fused_kernel<R, false, false><<<fgrid, kFuseThreads, fsm, s>>>(c);
      batch_fused_kernel<R, false, true><<<fgrid, kFuseThreads, fsm, s>>>(c);
    }
    batch_commit_plan_kernel<R><<<c.S, 1024, 0, s>>>(c);
    count_launch(5);
  }
  // the per-step path: one tile space over all live slots, strided by a persistent grid
  batch_tiles_kernel<R><<<1, 1024, 0, s>>>(c);
  if (c.grid_fields) batch_step_kernel<R, true><<<c.target_blocks, kStepThreads, smem, s>>>(c);
  else batch_step_kernel<R, false><<<c.target_blocks, kStepThreads, smem, s>>>(c);
  batch_plan_kernel<R><<<c.S, 1024, 0, s>>>(c, c.target_blocks);
  batch_prefix_kernel<R><<<sm_count() * 8, 256, 0, s>>>(c);
  batch_scatter_kernel<R><<<sm_count() * 4, 256, 0, s>>>(c);
  count_launch(5);
}

#endif

#if QED_PART(1)
size_t step_scalars_bytes(int precision) {
  return precision == QED_MIXED ? sizeof(StepScalars<float>) : sizeof(StepScalars<double>);
}

// grid of the multi-step kernels: every SM full, never more blocks than ledger partials
template <typename R, bool G, bool C>
static int fused_grid(int max_parts, size_t smem) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fused_kernel<R, G, C>, kFuseThreads, smem);
  return std::max(1, std::min(max_parts, sm_count() * std::max(b, 1)));
}

template <typename R>
int launch_fused(const StepArgs<R>& a, int K, bool commit, uint32_t* first_event, int max_parts, cudaStream_t s) {
  const size_t smem = (size_t)(a.tab.n_eta + a.tab.n_chi) * sizeof(R);
  const bool g = a.field.kind == QED_FIELD_GRID;
  int grid;
  if (!commit) {
    set_u32_kernel<<<1, 1, 0, s>>>(first_event, (uint32_t)K);
    if (g) {
      grid = fused_grid<R, true, false>(max_parts, smem);
      fused_kernel<R, true, false><<<grid, kFuseThreads, smem, s>>>(a, K, first_event);
    } else {
      grid = fused_grid<R, false, false>(max_parts, smem);
      fused_kernel<R, false, false><<<grid, kFuseThreads, smem, s>>>(a, K, first_event);
    }
    count_launch(2);
  } else {
    if (g) {
      grid = fused_grid<R, true, true>(max_parts, smem);
      fused_kernel<R, true, true><<<grid, kFuseThreads, smem, s>>>(a, K, first_event);
    } else {
      grid = fused_grid<R, false, true>(max_parts, smem);
      fused_kernel<R, false, true><<<grid, kFuseThreads, smem, s>>>(a, K, first_event);
    }
    count_launch(1);
  }
  return grid;
}

int fuse_max_steps() { return kMaxFuse; }

void launch_selftest_wait(uint32_t polls, uint32_t* bits, cudaStream_t s) {
  selftest_wait_kernel<<<1, 32, 0, s>>>(polls, bits);
  count_launch();
}

template <typename R>
void launch_finalize(const StepArgs<R>& a, int step_grid, cudaStream_t s) {
  plan_kernel<R><<<1, 1024, 0, s>>>(a, step_grid);
  prefix_kernel<R><<<sm_count() * 4, 256, 0, s>>>(a);
  scatter_kernel<R><<<sm_count() * 4, 256, 0, s>>>(a);
  count_launch(3);
}

#endif

#if QED_PART(3)
template <typename R>
void launch_init_tau(const SpeciesDev<R>& sp, int kind, uint64_t seed, uint64_t scen, cudaStream_t s) {
  init_tau_kernel<R><<<sm_count() * 4, 256, 0, s>>>(sp, kind, seed, scen);
  count_launch();
}

template <typename R>
void launch_eval(const TabDev<R>& tab, const FieldDev& f, int kind, double t, double wx0, double wv, size_t n,
                 const double* x, const double* y, const double* z, const double* ux, const double* uy,
                 const double* uz, double* oE, double* oB, double* op, double* oe, double* orate, cudaStream_t s) {
  eval_kernel<R><<<small_grid(n), 256, 0, s>>>(tab, f, kind, t, wx0, wv, n, x, y, z, ux, uy, uz, oE, oB, op, oe, orate);
  count_launch();
}

template <typename R>
void launch_sample(const TabDev<R>& tab, int which, size_t n, const double* param, const double* U, double* out,
                   int32_t* ok, cudaStream_t s) {
  sample_kernel<R><<<small_grid(n), 256, 0, s>>>(tab, which, n, param, U, out, ok);
  count_launch();
}

void launch_philox(size_t n, const uint64_t* ctr, uint64_t k0, uint64_t k1, uint64_t* out, cudaStream_t s) {
  philox_kernel<<<small_grid(n), 256, 0, s>>>(n, ctr, k0, k1, out);
  count_launch();
}

void launch_tau_convert(int precision, double* tau, size_t n, bool to_double, cudaStream_t s) {
  if (precision != QED_MIXED || n == 0) return;
  if (to_double) tau_to_double_kernel<float><<<small_grid(n), 256, 0, s>>>(tau, n);
  else tau_from_double_kernel<float><<<small_grid(n), 256, 0, s>>>(tau, n);
  count_launch();
}

template <typename R>
void launch_compact(const SpeciesDev<R>& sp, const SpeciesDev<R>& out, uint32_t* seg_count, uint32_t* seg_prefix,
                    cudaStream_t s) {
  compact_count_kernel<R><<<sm_count() * 4, 256, 0, s>>>(sp, seg_count);
  compact_scan_kernel<R><<<1, 1024, 0, s>>>(sp, seg_count, seg_prefix);
  compact_scatter_kernel<R><<<sm_count() * 4, 256, 0, s>>>(sp, out, seg_prefix);
  compact_finish_kernel<R><<<1, 1, 0, s>>>(sp, seg_prefix);
  count_launch(4);
}

// ----------------------------------------------------------------------------- weights, merging
template <typename R>
__global__ void fill_kernel(R* p, size_t n, R v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// Per-block FP64 partials of the physical totals: sum w, sum w * energy, sum w * momentum.
template <typename R>
__global__ void __launch_bounds__(256) totals_kernel(const SpeciesDev<R> sp, int massless, double* partials) {
  const uint32_t n = sp.cnt->n;
  double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (massless && Tau<R>::load(sp.tau + i).dead()) continue;
    const double u[3] = {(double)sp.ux[i], (double)sp.uy[i], (double)sp.uz[i]};
    const double w = sp.w ? (double)sp.w[i] : 1.0;
    const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    t[0] += w;
    t[1] += w * (massless ? sqrt(u2) : sqrt(1.0 + u2));
    for (int c = 0; c < 3; ++c) t[2 + c] += w * u[c];
  }
  __shared__ double s_t[8][5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < 5; ++c) {
    double v = t[c];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFull, v, off);
    if (lane == 0) s_t[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double v = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += s_t[q][threadIdx.x];
    partials[blockIdx.x * 5 + threadIdx.x] = v;
  }
}

// Group key of a photon for merging, or ~0 when it is not merged: position cell, cube-face
// direction bin and binary-exponent energy bin, from exact operations only (divisions, floor,
// frexp) in double, so that it equals the key any other IEEE double implementation computes.
__device__ uint64_t merge_key_dev(const double x[3], const double k[3], const MergeDev& M) {
  uint64_t cell = 0;
  for (int a = 2; a >= 0; --a) {
    const double c = floor((x[a] - M.origin[a]) / M.cell[a]);
    if (!(c >= 0.0 && c < (double)M.n_cells[a])) return ~0ull;
    cell = cell * (uint64_t)M.n_cells[a] + (uint64_t)c;
  }
  int ax = 0;
  for (int a = 1; a < 3; ++a)
    if (fabs(k[a]) > fabs(k[ax])) ax = a;
  const double m = fabs(k[ax]);
  if (!(m > 0.0)) return ~0ull;
  const int face = 2 * ax + (k[ax] < 0.0 ? 1 : 0);
  int fb[2], q = 0;
  for (int a = 0; a < 3; ++a) {
    if (a == ax) continue;
    int b = (int)floor((k[a] / m + 1.0) * 0.5 * M.n_face);
    b = b < 0 ? 0 : (b >= M.n_face ? M.n_face - 1 : b);
    fb[q++] = b;
  }
  const uint64_t dir = ((uint64_t)face * M.n_face + fb[0]) * M.n_face + fb[1];
  int e2 = 0;
  const double mant = frexp(sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]), &e2);
  int sub = (int)floor((mant - 0.5) * 2.0 * M.n_sub);
  if (sub >= M.n_sub) sub = M.n_sub - 1;
  const uint64_t en = (uint64_t)(e2 + 1100) * (uint64_t)M.n_sub + (uint64_t)sub;
  return (cell << 32) | (dir << 16) | en;
}

template <typename R>
__global__ void merge_key_kernel(const SpeciesDev<R> sp, MergeDev M, uint64_t* keys, uint32_t* idx, uint32_t N) {
  const uint32_t n = sp.cnt->n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    uint64_t key = ~0ull;
    if (i < n && !Tau<R>::load(sp.tau + i).dead()) {
      const double x[3] = {(double)sp.x[i], (double)sp.y[i], (double)sp.z[i]};
      const double k[3] = {(double)sp.ux[i], (double)sp.uy[i], (double)sp.uz[i]};
      key = merge_key_dev(x, k, M);
    }
    keys[i] = key;
    idx[i] = i;
  }
}

// One compare-exchange pass of a bitonic sort of (key, index) pairs (N a power of two): the
// result is ordered by key, and by index within a key.
__global__ void bitonic_pass_kernel(uint64_t* keys, uint32_t* idx, uint32_t N, uint32_t k, uint32_t j) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const uint32_t l = i ^ j;
    if (l <= i) continue;
    const bool asc = (i & k) == 0u;
    const uint64_t ka = keys[i], kb = keys[l];
    const uint32_t ia = idx[i], ib = idx[l];
    const bool greater = ka > kb || (ka == kb && ia > ib);
    if (greater == asc) {
      keys[i] = kb; keys[l] = ka;
      idx[i] = ib; idx[l] = ia;
    }
  }
}

// One thread per group (at the group's first sorted position): groups of at least min_group
// photons become two (the two lowest indices) that carry the group's weight, momentum and energy;
// the others become holes (tau = +inf) that compaction removes.
template <typename R>
__global__ void merge_groups_kernel(SpeciesDev<R> sp, MergeDev M, const uint64_t* keys, const uint32_t* idx, uint32_t N,
                                    int massless, unsigned long long* groups) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const uint64_t key = keys[p];
    if (key == ~0ull || (p > 0 && keys[p - 1] == key)) continue;
    uint32_t q = p + 1;
    while (q < N && keys[q] == key) ++q;
    if ((int)(q - p) < M.min_group) continue;
    double W = 0.0, E = 0.0, P[3] = {0.0, 0.0, 0.0}, X[3] = {0.0, 0.0, 0.0};
    for (uint32_t r = p; r < q; ++r) {
      const uint32_t i = idx[r];
      const double w = sp.w ? (double)sp.w[i] : 1.0;
      const double k[3] = {(double)sp.ux[i], (double)sp.uy[i], (double)sp.uz[i]};
      const double x[3] = {(double)sp.x[i], (double)sp.y[i], (double)sp.z[i]};
      const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
      W += w;
      E += w * (massless ? sqrt(k2) : sqrt(1.0 + k2));
      for (int c = 0; c < 3; ++c) { P[c] += w * k[c]; X[c] += w * x[c]; }
    }
    // both members get energy E/W; massive ones sit on the mass shell, |u|^2 = (E/W)^2 - 1
    const double et = E / W, mv[3] = {P[0] / W, P[1] / W, P[2] / W};
    const double m2 = mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
    const double d2 = (massless ? et * et : et * et - 1.0) - m2;
    const double dl = d2 > 0.0 ? sqrt(d2) : 0.0;
    int ax = 0;
    for (int c = 1; c < 3; ++c)
      if (fabs(mv[c]) < fabs(mv[ax])) ax = c;
    double e[3] = {0.0, 0.0, 0.0};
    e[ax] = 1.0;
    double dv[3] = {mv[1] * e[2] - mv[2] * e[1], mv[2] * e[0] - mv[0] * e[2], mv[0] * e[1] - mv[1] * e[0]};
    const double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    if (dn > 0.0) {
      for (int c = 0; c < 3; ++c) dv[c] *= dl / dn;
    } else {
      for (int c = 0; c < 3; ++c) dv[c] = 0.0;
      dv[ax] = dl;
    }
    for (int t = 0; t < 2; ++t) {
      const uint32_t i = idx[p + t];
      const double sg = t == 0 ? 1.0 : -1.0;
      sp.ux[i] = (R)(mv[0] + sg * dv[0]); sp.uy[i] = (R)(mv[1] + sg * dv[1]); sp.uz[i] = (R)(mv[2] + sg * dv[2]);
      sp.x[i] = (R)(X[0] / W); sp.y[i] = (R)(X[1] / W); sp.z[i] = (R)(X[2] / W);
      if (sp.w) sp.w[i] = (R)(0.5 * W);
    }
    for (uint32_t r = p + 2; r < q; ++r) Tau<R>::infinite().store(sp.tau + idx[r]);
    atomicAdd(&sp.cnt->n_dead, q - p - 2);
    atomicAdd(groups, 1ull);
  }
}

template <typename R>
void launch_fill(R* p, size_t n, R v, cudaStream_t s) {
  if (!n) return;
  fill_kernel<R><<<sm_count() * 4, 256, 0, s>>>(p, n, v);
  count_launch();
}

template <typename R>
void launch_totals(const SpeciesDev<R>& sp, int massless, double* partials, int blocks, cudaStream_t s) {
  totals_kernel<R><<<blocks, 256, 0, s>>>(sp, massless, partials);
  count_launch();
}

template <typename R>
void launch_merge(const SpeciesDev<R>& sp, const MergeDev& m, uint64_t* keys, uint32_t* idx, uint32_t N,
                  int massless, unsigned long long* groups, cudaStream_t s) {
  const int grid = sm_count() * 8;
  merge_key_kernel<R><<<grid, 256, 0, s>>>(sp, m, keys, idx, N);
  int launches = 1;
  for (uint32_t k = 2; k <= N; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      bitonic_pass_kernel<<<grid, 256, 0, s>>>(keys, idx, N, k, j);
      ++launches;
    }
  merge_groups_kernel<R><<<grid, 256, 0, s>>>(sp, m, keys, idx, N, massless, groups);
  count_launch(launches + 1);
}

#endif

#if QED_PART(1)
#define QED_INSTANTIATE_STEP(R)                                                                                  \
  template void launch_step<R>(const StepArgs<R>&, int, int, size_t, cudaStream_t);                              \
  template void launch_finalize<R>(const StepArgs<R>&, int, cudaStream_t);                                       \
  template int launch_fused<R>(const StepArgs<R>&, int, bool, uint32_t*, int, cudaStream_t);
QED_INSTANTIATE_STEP(float)
QED_INSTANTIATE_STEP(double)
#endif
#if QED_PART(2)
template void launch_batch_step<float>(const BatchCtl<float>&, int, int, cudaStream_t);
template void launch_batch_step<double>(const BatchCtl<double>&, int, int, cudaStream_t);
#endif
#if QED_PART(3)
#define QED_INSTANTIATE(R)                                                                                       \
  template void launch_init_tau<R>(const SpeciesDev<R>&, int, uint64_t, uint64_t, cudaStream_t);                 \
  template void launch_eval<R>(const TabDev<R>&, const FieldDev&, int, double, double, double, size_t,           \
                               const double*, const double*, const double*, const double*, const double*,        \
                               const double*, double*, double*, double*, double*, double*, cudaStream_t);        \
  template void launch_sample<R>(const TabDev<R>&, int, size_t, const double*, const double*, double*, int32_t*, \
                                 cudaStream_t);                                                                  \
  template void launch_compact<R>(const SpeciesDev<R>&, const SpeciesDev<R>&, uint32_t*, uint32_t*, cudaStream_t); \
  template void launch_fill<R>(R*, size_t, R, cudaStream_t);                                                     \
  template void launch_totals<R>(const SpeciesDev<R>&, int, double*, int, cudaStream_t);                         \
  template void launch_merge<R>(const SpeciesDev<R>&, const MergeDev&, uint64_t*, uint32_t*, uint32_t, int,        \
                                unsigned long long*, cudaStream_t);
QED_INSTANTIATE(float)
QED_INSTANTIATE(double)
#endif

}  // namespace qedlib
