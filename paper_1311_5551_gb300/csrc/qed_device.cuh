// qed_device.cuh -- per-particle device functions of the QED Monte-Carlo step (Sec. 3).
// Templated on the arithmetic type R (float for the mixed path, double for the FP64 path).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qed_internal.h"

namespace qedlib {

template <typename R> struct Num;
// The FP64 path uses correctly rounded operations throughout.  The mixed path's per-particle
// push uses the hardware approximations where the FP32 result needs no more (a few ulp against a
// 1e-5 relative budget): reciprocal square roots, approximate division by quantities >= 1, and
// the fast carrier sine/cosine of arguments reduced to a few radians.
template <> struct Num<float> {
  static __device__ __forceinline__ float sqrt_(float v) { return sqrtf(v); }
  static __device__ __forceinline__ float log_(float v) { return logf(v); }
  static __device__ __forceinline__ float exp_(float v) { return expf(v); }
  static __device__ __forceinline__ void sincos_(float v, float* s, float* c) { sincosf(v, s, c); }
  static __device__ __forceinline__ float sinpi_(float v) { return sinpif(v); }
  static __device__ __forceinline__ float pow_(float a, float b) { return powf(a, b); }
  // hot-path forms
  static __device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ float rsqrt_(float v) { return rsqrtf(v); }
  static __device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float sqrt_pos_(float v) { return v * rsqrtf(v); }  // v > 0
  static __device__ __forceinline__ void carrier_(float v, float* s, float* c) { __sincosf(v, s, c); }
  static __device__ __forceinline__ float sin_env_(float v) { return __sinf(v); }
  // table coordinates and values: ln of eta or chi (absolute error < 4e-7) and exp of the
  // interpolated ln h or ln T (relative error < 1e-5 down to the FP32 underflow)
  static __device__ __forceinline__ float log_tab_(float v) { return __logf(v); }
  static __device__ __forceinline__ float exp_tab_(float v) { return __expf(v); }
  // a^b for a > 0 off the tables' ends (the chi^{-1/3} continuation of T)
  static __device__ __forceinline__ float pow_tab_(float a, float b) { return __expf(b * __logf(a)); }
  // sqrt(v) and 1/sqrt(v) for v >= 1 (gamma and its inverse)
  static __device__ __forceinline__ void root_inv_(float v, float& r, float& ir) { ir = rsqrtf(v); r = v * ir; }
};
template <> struct Num<double> {
  static __device__ __forceinline__ double sqrt_(double v) { return sqrt(v); }
  static __device__ __forceinline__ double log_(double v) { return log(v); }
  static __device__ __forceinline__ double exp_(double v) { return exp(v); }
  static __device__ __forceinline__ void sincos_(double v, double* s, double* c) { sincos(v, s, c); }
  static __device__ __forceinline__ double sinpi_(double v) { return sinpi(v); }
  static __device__ __forceinline__ double pow_(double a, double b) { return pow(a, b); }
  static __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
  static __device__ __forceinline__ double rsqrt_(double v) { return 1.0 / sqrt(v); }
  static __device__ __forceinline__ double div_(double a, double b) { return a / b; }
  static __device__ __forceinline__ double sqrt_pos_(double v) { return sqrt(v); }
  static __device__ __forceinline__ void carrier_(double v, double* s, double* c) { sincos(v, s, c); }
  static __device__ __forceinline__ double sin_env_(double v) { return sin(v); }
  static __device__ __forceinline__ double log_tab_(double v) { return log(v); }
  static __device__ __forceinline__ double exp_tab_(double v) { return exp(v); }
  static __device__ __forceinline__ double pow_tab_(double a, double b) { return pow(a, b); }
  static __device__ __forceinline__ void root_inv_(double v, double& r, double& ir) { r = sqrt(v); ir = 1.0 / r; }
};

constexpr double kAlpha = 7.2973525693e-3;           // fine-structure constant
constexpr double kSqrt3 = 1.7320508075688772;
constexpr double kTwoPi = 6.283185307179586;
constexpr double kPi = 3.141592653589793;
// lambda_gamma = (sqrt3 alpha c/lambda_c)(eta/gamma) h = (sqrt3 alpha/2pi)(eta/gamma) h, with
// lambda_c = h/(m c) the Compton wavelength, in units of m c^2/hbar (eq. rate_photons)
constexpr double kRatePhoton = kSqrt3 * kAlpha / kTwoPi;

// ------------------------------------------------------------------ Philox4x64-10
// Counter-based generator of Salmon, Moraes, Dror & Shaw (SC'11), 10 rounds.
__device__ __forceinline__ void philox4x64(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t a0 = c[0], a2 = c[2];
    const uint64_t lo0 = 0xD2E7470EE14C6C93ull * a0, hi0 = __umul64hi(0xD2E7470EE14C6C93ull, a0);
    const uint64_t lo1 = 0xCA5A826395121157ull * a2, hi1 = __umul64hi(0xCA5A826395121157ull, a2);
    c[0] = hi1 ^ c[1] ^ k0;
    c[1] = lo1;
    c[2] = hi0 ^ c[3] ^ k1;
    c[3] = lo0;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
}
// (m + 1/2) 2^-52 with m the top 52 bits: strictly inside (0, 1) and exact in double
__device__ __forceinline__ double u01(uint64_t w) { return ((double)(w >> 12) + 0.5) * 0x1.0p-52; }

// Stream layout: key (seed, scenario), counter (id, step, species kind, purpose 0 event / 1 init)
__device__ __forceinline__ void draw4(uint64_t seed, uint64_t scen, uint64_t id, uint64_t step, uint64_t kind,
                                      uint64_t purpose, double U[4]) {
  uint64_t c[4] = {id, step, kind, purpose};
  philox4x64(c, seed, scen);
#pragma unroll
  for (int i = 0; i < 4; ++i) U[i] = u01(c[i]);
}

// ------------------------------------------------------------------ TMA bulk copies (sm_90+)
// 1-D bulk copies global -> shared completed on an mbarrier (transaction-count based).
// Requirements (checked by the callers' layout): both addresses 16-byte aligned, size a
// multiple of 16 bytes.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// One poll that may suspend the thread until the phase completes or hint_ns nanoseconds pass
// (the suspended warp takes no issue slots from the warps that have work).
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return done != 0;
}
// Bounded wait: gives up after `limit` polls, each suspending for at most kPollHintNs, so a wait
// that can never end costs at most limit * kPollHintNs of time.
constexpr uint32_t kPollHintNs = 20000;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  if (mbar_try_wait(bar, parity)) return true;
  for (uint32_t it = 1; it < limit; ++it)
    if (mbar_try_wait_hint(bar, parity, kPollHintNs)) return true;
  return false;
}
// Orders this thread's view of earlier generic-proxy shared-memory accesses (made visible to it
// by a barrier) before its subsequent async-proxy (bulk copy) writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ------------------------------------------------------------------ per-step field scalars
template <typename R>
struct StepScalars {
  R E[3], B[3];    // uniform / rotating field at t_n
  R phi_ref;       // plane wave: omega (t_n - x_w(t_n)) - phi_start (phase at x_rel = 0)
  R phi_ref_mod;   // the same reduced to [-pi, pi] (carrier)
  R omega, E0, inv_len, len;
  int kind;
  // grid gather
  const R* grid;
  size_t gN;       // values per component
  int gn[3], shape;
  R gorg[3], ginv[3];
};

// FP64 per-step quantities (one thread per block).
template <typename R>
__device__ void make_scalars(const FieldDev& f, double t, double win_x0, double win_v, StepScalars<R>& S) {
  S.kind = f.kind;
  for (int c = 0; c < 3; ++c) { S.E[c] = (R)0; S.B[c] = (R)0; }
  S.omega = (R)f.omega;
  S.E0 = (R)f.E0;
  S.len = (R)f.phi_len;
  S.inv_len = f.phi_len > 0.0 ? (R)(1.0 / f.phi_len) : (R)0;
  S.phi_ref = (R)0;
  S.phi_ref_mod = (R)0;
  S.grid = nullptr;
  if (f.kind == QED_FIELD_GRID) {
    S.grid = static_cast<const R*>(f.grid);
    S.shape = f.shape;
    S.gN = (size_t)f.n[0] * (size_t)f.n[1] * (size_t)f.n[2];
    for (int c = 0; c < 3; ++c) {
      S.gn[c] = f.n[c];
      S.gorg[c] = (R)f.origin[c];
      S.ginv[c] = (R)(1.0 / f.spacing[c]);
    }
  } else if (f.kind == QED_FIELD_UNIFORM) {
    for (int c = 0; c < 3; ++c) { S.E[c] = (R)f.E[c]; S.B[c] = (R)f.B[c]; }
  } else if (f.kind == QED_FIELD_ROTATING_E) {
    double s, c;
    sincos(f.omega * t + f.phase0, &s, &c);
    S.E[0] = (R)(f.E0 * c);
    S.E[1] = (R)(f.E0 * s);
  } else {
    const double xw = win_x0 + win_v * t;
    const double ph = f.omega * (t - xw) - f.phi_start;
    S.phi_ref = (R)ph;
    S.phi_ref_mod = (R)(ph - kTwoPi * rint(ph / kTwoPi));
  }
}

// ------------------------------------------------------------------ grid gather (Sec. 3.2)
// Node weights along one axis for a particle at continuous node index s: W = 2 (cloud-in-cell,
// nodes i0, i0 + 1) or W = 3 (triangular-shaped cloud, nodes i0 .. i0 + 2 around the nearest).
template <typename R, int W>
struct AxisWeights {
  int i0;
  R w[W];
};

template <typename R, int W>
__device__ __forceinline__ AxisWeights<R, W> axis_weights(R s) {
  AxisWeights<R, W> a;
  if (W == 2) {
    const R f = floor(s);
    const R d = s - f;
    a.i0 = (int)f;
    a.w[0] = (R)1 - d;
    a.w[1] = d;
  } else {
    const R m = rint(s);
    const R d = s - m;  // in [-1/2, 1/2]
    a.i0 = (int)m - 1;
    const R l = (R)0.5 - d, r = (R)0.5 + d;
    a.w[0] = (R)0.5 * l * l;
    a.w[1] = (R)0.75 - d * d;
    a.w[W - 1] = (R)0.5 * r * r;
  }
  return a;
}

// One component: sum of w_x w_y w_z * value over the stencil nodes that exist.
template <typename R, int W>
__device__ __forceinline__ R gather_component(const R* __restrict__ G, const int n[3], const AxisWeights<R, W>& ax,
                                              const AxisWeights<R, W>& ay, const AxisWeights<R, W>& az) {
  R v = (R)0;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const int iz = az.i0 + k;
    if (iz < 0 || iz >= n[2]) continue;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const int iy = ay.i0 + j;
      if (iy < 0 || iy >= n[1]) continue;
      const R wzy = az.w[k] * ay.w[j];
      const R* row = G + ((size_t)iz * (size_t)n[1] + (size_t)iy) * (size_t)n[0];
#pragma unroll
      for (int i = 0; i < W; ++i) {
        const int ix = ax.i0 + i;
        if (ix < 0 || ix >= n[0]) continue;
        v = Num<R>::fma_(wzy * ax.w[i], __ldg(row + ix), v);
      }
    }
  }
  return v;
}

// E_c is staggered half a cell along axis c, cB_c along the two other axes (Yee).
template <typename R, int W>
__device__ __forceinline__ void gather_fields(const StepScalars<R>& S, const R s[3], R E[3], R B[3]) {
  AxisWeights<R, W> node[3], half[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    node[a] = axis_weights<R, W>(s[a]);
    half[a] = axis_weights<R, W>(s[a] - (R)0.5);
  }
  E[0] = gather_component<R, W>(S.grid + 0 * S.gN, S.gn, half[0], node[1], node[2]);
  E[1] = gather_component<R, W>(S.grid + 1 * S.gN, S.gn, node[0], half[1], node[2]);
  E[2] = gather_component<R, W>(S.grid + 2 * S.gN, S.gn, node[0], node[1], half[2]);
  B[0] = gather_component<R, W>(S.grid + 3 * S.gN, S.gn, node[0], half[1], half[2]);
  B[1] = gather_component<R, W>(S.grid + 4 * S.gN, S.gn, half[0], node[1], half[2]);
  B[2] = gather_component<R, W>(S.grid + 5 * S.gN, S.gn, half[0], half[1], node[2]);
}

template <typename R>
__device__ __forceinline__ void grid_field_at(const StepScalars<R>& S, R x, R y, R z, R E[3], R B[3]) {
  E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = (R)0;
  const R s[3] = {(x - S.gorg[0]) * S.ginv[0], (y - S.gorg[1]) * S.ginv[1], (z - S.gorg[2]) * S.ginv[2]};
  // far outside nothing contributes; this also keeps the node indices within int range
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (!(s[a] > (R)-3 && s[a] < (R)S.gn[a] + (R)2)) return;
  if (S.shape == 1) gather_fields<R, 2>(S, s, E, B);
  else gather_fields<R, 3>(S, s, E, B);
}

// Fields at the particle (position relative to the window) at t_n.  G: the caller is the
// grid-capable instantiation of the step (the gather's stencil costs registers, so kernels that
// never see a grid field are compiled without it).
// What field_at found: no field (the push and the quantum parameter are identities), a general
// field, or a plane wave along +x (E perpendicular to x, cB = xhat x E) of magnitude |E|.
enum FieldCase { kNoField = 0, kGeneralField = 1, kPlaneWave = 2 };

template <typename R, bool G>
__device__ __forceinline__ int field_at(const StepScalars<R>& S, R xrel, R y, R z, R E[3], R B[3], R& amp) {
  if (S.kind == QED_FIELD_UNIFORM || S.kind == QED_FIELD_ROTATING_E) {
#pragma unroll
    for (int c = 0; c < 3; ++c) { E[c] = S.E[c]; B[c] = S.B[c]; }
    return kGeneralField;
  }
  if constexpr (G) {
    if (S.kind == QED_FIELD_GRID) {
      grid_field_at<R>(S, xrel, y, z, E, B);
      return kGeneralField;
    }
  }
  E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = (R)0;
  R env = (R)1;
  if (S.len > (R)0) {
    const R phi = Num<R>::fma_(-S.omega, xrel, S.phi_ref);
    if (!(phi > (R)0) || !(phi < S.len)) return kNoField;
    const R s = Num<R>::sin_env_((R)kPi * (phi * S.inv_len));
    env = s * s;
  }
  R sn, cs;
  Num<R>::carrier_(Num<R>::fma_(-S.omega, xrel, S.phi_ref_mod), &sn, &cs);
  const R a = S.E0 * env;
  if (S.kind == QED_FIELD_PLANE_LP) {
    E[1] = a * cs;
    B[2] = a * cs;
    amp = fabs(E[1]);
  } else {
    E[1] = a * cs;
    E[2] = a * sn;
    B[1] = -a * sn;
    B[2] = a * cs;
    amp = a;
  }
  return kPlaneWave;
}

// ------------------------------------------------------------------ push, eta, chi
// Boris push u^{n-1/2} -> u^{n+1/2} (half electric kick, rotation with the gamma of the
// half-kicked momentum, half electric kick), Vlasov LHS of Sec. 2.3.
template <typename R>
__device__ __forceinline__ void boris(R q, R dt, const R E[3], const R B[3], R u[3]) {
  using N = Num<R>;
  const R hq = (R)0.5 * q * dt;
  const R m0 = N::fma_(hq, E[0], u[0]), m1 = N::fma_(hq, E[1], u[1]), m2 = N::fma_(hq, E[2], u[2]);
  const R ig = N::rsqrt_(N::fma_(m0, m0, N::fma_(m1, m1, N::fma_(m2, m2, (R)1))));
  const R hb = hq * ig;
  const R t0 = hb * B[0], t1 = hb * B[1], t2 = hb * B[2];
  const R f = N::div_((R)2, N::fma_(t0, t0, N::fma_(t1, t1, N::fma_(t2, t2, (R)1))));
  const R s0 = f * t0, s1 = f * t1, s2 = f * t2;
  // p = m + m x t, then u = m + p x s + the second half kick
  const R p0 = m0 + N::fma_(m1, t2, -(m2 * t1)), p1 = m1 + N::fma_(m2, t0, -(m0 * t2)),
          p2 = m2 + N::fma_(m0, t1, -(m1 * t0));
  u[0] = N::fma_(hq, E[0], m0 + N::fma_(p1, s2, -(p2 * s1)));
  u[1] = N::fma_(hq, E[1], m1 + N::fma_(p2, s0, -(p0 * s2)));
  u[2] = N::fma_(hq, E[2], m2 + N::fma_(p0, s1, -(p1 * s0)));
}

// |v|^2 and cross products with explicit multiply-adds (no implicit contraction is compiled)
template <typename R>
__device__ __forceinline__ R dot3(const R a[3], const R b[3]) {
  return Num<R>::fma_(a[0], b[0], Num<R>::fma_(a[1], b[1], a[2] * b[2]));
}
template <typename R>
__device__ __forceinline__ void cross3(const R a[3], const R b[3], R c[3]) {
  c[0] = Num<R>::fma_(a[1], b[2], -(a[2] * b[1]));
  c[1] = Num<R>::fma_(a[2], b[0], -(a[0] * b[2]));
  c[2] = Num<R>::fma_(a[0], b[1], -(a[1] * b[0]));
}

// eta^2 = (gamma E + u x cB)^2 - (u.E)^2 = E^2 + |u x E|^2 + 2 gamma E.(u x cB) + |u x cB|^2
template <typename R>
__device__ __forceinline__ R eta_of(const R u[3], R gamma, const R E[3], const R B[3]) {
  R ue[3], ub[3];
  cross3<R>(u, E, ue);
  cross3<R>(u, B, ub);
  const R e2 = (dot3<R>(E, E) + dot3<R>(ue, ue)) + Num<R>::fma_((R)2 * gamma, dot3<R>(E, ub), dot3<R>(ub, ub));
  return e2 > (R)0 ? Num<R>::sqrt_pos_(e2) : (R)0;
}

// chi (Sec. 2, half the usual chi_gamma): 4 chi^2 = |k x E|^2 + 2 eps E.(k x cB) + |k x cB|^2
template <typename R>
__device__ __forceinline__ R chi_of(const R k[3], R eps, const R E[3], const R B[3]) {
  R ke[3], kb[3];
  cross3<R>(k, E, ke);
  cross3<R>(k, B, kb);
  const R c2 = dot3<R>(ke, ke) + Num<R>::fma_((R)2 * eps, dot3<R>(E, kb), dot3<R>(kb, kb));
  return c2 > (R)0 ? (R)0.5 * Num<R>::sqrt_pos_(c2) : (R)0;
}

// In a plane wave along +x (cB = xhat x E, E perpendicular to x) the invariants reduce to
// eta = (gamma - u_x)|E| and chi = (eps - k_x)|E|/2 exactly; gamma - u_x is written as
// (1 + u_perp^2)/(gamma + u_x) when u_x > 0, so co-propagating particles lose no digits.
template <typename R>
__device__ __forceinline__ R eta_plane(const R u[3], R gamma, R amp) {
  using N = Num<R>;
  const R d = u[0] > (R)0 ? N::div_(N::fma_(u[1], u[1], N::fma_(u[2], u[2], (R)1)), gamma + u[0]) : gamma - u[0];
  return d * amp;
}
template <typename R>
__device__ __forceinline__ R chi_plane(const R k[3], R eps, R amp) {
  using N = Num<R>;
  const R d = k[0] > (R)0 ? N::div_(N::fma_(k[1], k[1], k[2] * k[2]), eps + k[0]) : eps - k[0];
  return (R)0.5 * d * amp;
}

// The quantum parameters for the case field_at reported.
template <typename R>
__device__ __forceinline__ R eta_for(int fc, const R u[3], R gamma, const R E[3], const R B[3], R amp) {
  if (fc == kPlaneWave) return eta_plane<R>(u, gamma, amp);
  return fc == kNoField ? (R)0 : eta_of<R>(u, gamma, E, B);
}
template <typename R>
__device__ __forceinline__ R chi_for(int fc, const R k[3], R eps, const R E[3], const R B[3], R amp) {
  if (fc == kPlaneWave) return chi_plane<R>(k, eps, amp);
  return fc == kNoField ? (R)0 : chi_of<R>(k, eps, E, B);
}

// ------------------------------------------------------------------ field classes
// The step's kernels are compiled per field class, chosen per tile (uniform across a warp):
// any field (field_at, the general push and invariants), or a plane wave along +x, linearly
// (E = (0, e, 0), cB = (0, 0, e)) or circularly polarised (E = (0, ey, ez), cB = (0, -ez, ey)),
// where the zero components are dropped from the push and eta, chi take their closed forms.
// On the components that are not zero they compute what field_at, boris and eta_for / chi_for
// compute, operation for operation (a zero component only adds exact zeros there).
enum FieldClass { kFieldAny = 0, kFieldLP = 1, kFieldCP = 2 };

// The plane wave at the particle (as field_at): false where the envelope vanishes.
template <typename R, int FC>
__device__ __forceinline__ bool plane_at(const StepScalars<R>& S, R xrel, R& ey, R& ez, R& amp) {
  R env = (R)1;
  if (S.len > (R)0) {
    const R phi = Num<R>::fma_(-S.omega, xrel, S.phi_ref);
    if (!(phi > (R)0) || !(phi < S.len)) return false;
    const R s = Num<R>::sin_env_((R)kPi * (phi * S.inv_len));
    env = s * s;
  }
  R sn, cs;
  Num<R>::carrier_(Num<R>::fma_(-S.omega, xrel, S.phi_ref_mod), &sn, &cs);
  const R a = S.E0 * env;
  ey = a * cs;
  if (FC == kFieldLP) {
    ez = (R)0;
    amp = fabs(ey);
  } else {
    ez = a * sn;
    amp = a;
  }
  return true;
}

// boris() for a plane wave along +x: E = (0, ey, ez), cB = (0, -ez, ey) (LP: ez = 0).
template <typename R, int FC>
__device__ __forceinline__ void boris_plane(R q, R dt, R ey, R ez, R u[3]) {
  using N = Num<R>;
  const R hq = (R)0.5 * q * dt;
  const R m0 = u[0], m1 = N::fma_(hq, ey, u[1]);
  const R m2 = FC == kFieldLP ? u[2] : N::fma_(hq, ez, u[2]);
  const R ig = N::rsqrt_(N::fma_(m0, m0, N::fma_(m1, m1, N::fma_(m2, m2, (R)1))));
  const R hb = hq * ig;
  if (FC == kFieldLP) {
    const R t2 = hb * ey;
    const R f = N::div_((R)2, N::fma_(t2, t2, (R)1));
    const R s2 = f * t2;
    const R p0 = m0 + m1 * t2, p1 = m1 - m0 * t2;
    u[0] = m0 + p1 * s2;
    u[1] = N::fma_(hq, ey, m1 - p0 * s2);
    u[2] = m2;
  } else {
    const R t1 = hb * -ez, t2 = hb * ey;
    const R f = N::div_((R)2, N::fma_(t1, t1, N::fma_(t2, t2, (R)1)));
    const R s1 = f * t1, s2 = f * t2;
    const R p0 = m0 + N::fma_(m1, t2, -(m2 * t1)), p1 = m1 - m0 * t2, p2 = m2 + m0 * t1;
    u[0] = m0 + N::fma_(p1, s2, -(p2 * s1));
    u[1] = N::fma_(hq, ey, m1 - p0 * s2);
    u[2] = N::fma_(hq, ez, m2 + p0 * s1);
  }
}

// ------------------------------------------------------------------ table look-ups (Sec. 3)
// Cell and weight on a uniform grid in ln v; oor = -1 below, +1 above, 0 inside.  Below the
// grid the first node is taken (w = 0), above it the last (w = 1), written as clamps rather than
// branches (the same results: a cell index of a position below 0 truncates to 0).
template <typename R>
__device__ __forceinline__ void grid_pos(R lnv, R lo, R inv_d, int n, int& i, R& w, int& oor) {
  const R s = (lnv - lo) * inv_d;
  oor = s < (R)0 ? -1 : (s > (R)(n - 1) ? 1 : 0);
  const R sc = s > (R)0 ? s : (R)0;  // also maps NaN to 0
  i = min((int)sc, n - 2);
  const R d = sc - (R)i;
  w = d < (R)1 ? d : (R)1;
}

// h(eta): linear interpolation in (ln eta, ln h); clamped above the table.
template <typename R>
__device__ __forceinline__ R lookup_h(const TabDev<R>& T, const R* lnh, R eta, int& oor) {
  int i; R w;
  grid_pos(Num<R>::log_tab_(eta), T.ln_eta_min, T.inv_d_eta, T.n_eta, i, w, oor);
  return Num<R>::exp_tab_(Num<R>::fma_(w, lnh[i + 1], ((R)1 - w) * lnh[i]));
}

// T above the table: the chi^{-1/3} continuation of App. B (FP32: exp and ln intrinsics, about
// 1e-6 relative; FP64: pow).
template <typename R>
__device__ __forceinline__ R T_above(const TabDev<R>& T, R chi) {
  return T.T_at_chi_max * Num<R>::pow_tab_(chi / T.chi_max, (R)(-1.0 / 3.0));
}

// T(chi): zero below the table, chi^{-1/3} above it (App. B), log-log interpolation inside.
template <typename R>
__device__ __forceinline__ R lookup_T(const TabDev<R>& T, const R* lnT, R chi, int& oor) {
  oor = 0;
  if (!(chi >= T.chi_min)) return (R)0;
  if (chi > T.chi_max) { oor = 1; return T_above<R>(T, chi); }
  int i, o; R w;
  grid_pos(Num<R>::log_tab_(chi), T.ln_chi_min, T.inv_d_chi, T.n_chi, i, w, o);
  return Num<R>::exp_tab_(Num<R>::fma_(w, lnT[i + 1], ((R)1 - w) * lnT[i]));
}

template <typename R>
__device__ __forceinline__ R xi_node(const TabDev<R>& T, int r, int j) {
  const R zlo = __ldg(T.zeta_lo + r), zhi = __ldg(T.zeta_hi + r);
  const R z = zlo + (R)j * (zhi - zlo) / (R)(T.n_xi - 1);
  return (R)1 / ((R)1 + Num<R>::exp_(-z));
}

// Invert one P_chi row: xi linear in P between the bracketing nodes; the complement Q is used
// when U > 1/2 (the same interpolation, precise near P = 1).
template <typename R>
__device__ R invert_xi_row(const TabDev<R>& T, int r, R U, R V) {
  const int n = T.n_xi;
  const R* P = T.P + (size_t)r * n;
  const R* Q = T.Q + (size_t)r * n;
  if (U <= __ldg(P)) return xi_node(T, r, 0);
  if (V <= __ldg(Q + n - 1)) return xi_node(T, r, n - 1);
  int lo = 0, hi = n - 1;
  R frac;
  if (U <= (R)0.5) {
    while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (__ldg(P + mid) < U) lo = mid; else hi = mid; }
    const R p0 = __ldg(P + lo), p1 = __ldg(P + lo + 1);
    frac = (U - p0) / (p1 - p0);
  } else {
    while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (__ldg(Q + mid) > V) lo = mid; else hi = mid; }
    const R q0 = __ldg(Q + lo), q1 = __ldg(Q + lo + 1);
    frac = (q0 - V) / (q0 - q1);
  }
  const R x0 = xi_node(T, r, lo), x1 = xi_node(T, r, lo + 1);
  return x0 + frac * (x1 - x0);
}

// Photon energy fraction xi = 2chi/eta (Sec. 3); false when U is below the cut-off.
template <typename R>
__device__ bool sample_xi(const TabDev<R>& T, R eta, R U, R V, R& xi) {
  int i, o; R w;
  grid_pos(Num<R>::log_(eta), T.ln_eta_min, T.inv_d_eta, T.n_eta, i, w, o);
  const int n = T.n_xi;
  const R pcut = ((R)1 - w) * __ldg(T.P + (size_t)i * n) + w * __ldg(T.P + (size_t)(i + 1) * n);
  if (U < pcut) return false;
  R x = ((R)1 - w) * invert_xi_row(T, i, U, V);
  if (w > (R)0) x += w * invert_xi_row(T, i + 1, U, V);
  if (o < 0) x *= eta / T.eta_min;  // classical scaling below the table
  if (x > (R)1) x = (R)1;
  xi = x;
  return true;
}

template <typename R>
__device__ R invert_f_row(const TabDev<R>& T, int r, R V) {
  const int n = T.n_f;
  const R* P = T.Pf + (size_t)r * n;
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (__ldg(P + mid) < V) lo = mid; else hi = mid; }
  const R p0 = __ldg(P + lo), p1 = __ldg(P + lo + 1);
  const R frac = (V - p0) / (p1 - p0);
  const R f0 = (R)0.5 * (R)lo / (R)(n - 1), f1 = (R)0.5 * (R)(lo + 1) / (R)(n - 1);
  return f0 + frac * (f1 - f0);
}

// Positron energy fraction f (Sec. 3, App. B): U < 1/2 maps to f <= 1/2 through V = 2U,
// U >= 1/2 to f >= 1/2 through V = 2(1 - U).
template <typename R>
__device__ R sample_f(const TabDev<R>& T, R chi, R U, R Vc) {
  int i, o; R w;
  grid_pos(Num<R>::log_(chi), T.ln_chi_min, T.inv_d_chi, T.n_chi, i, w, o);
  const bool lower = U < (R)0.5;
  const R V = lower ? (R)2 * U : (R)2 * Vc;
  R fh = ((R)1 - w) * invert_f_row(T, i, V);
  if (w > (R)0) fh += w * invert_f_row(T, i + 1, V);
  return lower ? fh : (R)1 - fh;
}

// ------------------------------------------------------------------ optical depth storage
// The remaining optical depth tau occupies 8 bytes per particle.  FP64 path: a double.  Mixed
// path: a compensated pair of floats (hi, lo) with tau = hi + lo (about 48 significant bits),
// advanced with error-free transformations, so the hot loop issues no FP64 instruction (FP64
// and float<->double conversions share GB300's slow FP64 pipe).  A converted photon is marked
// by tau = +inf (hi = +inf for the pair).
template <typename R> struct Tau;
template <> struct Tau<double> {
  double v;
  static __device__ __forceinline__ Tau load(const double* p) { return Tau{*p}; }
  static __device__ __forceinline__ Tau from_stored(double v) { return Tau{v}; }
  __device__ __forceinline__ void store(double* p) const { *p = v; }
  __device__ __forceinline__ void sub(double d) { v -= d; }
  // tau <= 0 as an integer sign test on the IEEE bits: +0 has all bits clear, every negative
  // value (-0 included) has the sign bit set
  __device__ __forceinline__ bool used_up() const { return __double_as_longlong(v) <= 0; }
  __device__ __forceinline__ bool dead() const { return __double_as_longlong(v) == 0x7ff0000000000000ll; }
  static __device__ __forceinline__ Tau fresh(double x) { return Tau{x}; }
  static __device__ __forceinline__ Tau infinite() { return Tau{__longlong_as_double(0x7ff0000000000000ll)}; }
  static __device__ __forceinline__ Tau one() { return Tau{1.0}; }
};
template <> struct Tau<float> {
  float hi, lo;
  static __device__ __forceinline__ Tau load(const double* p) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    return Tau{v.x, v.y};
  }
  // the stored 8 bytes held in a register: hi is the first (low-address, low-order) word
  static __device__ __forceinline__ Tau from_stored(double v) {
    return Tau{__int_as_float(__double2loint(v)), __int_as_float(__double2hiint(v))};
  }
  __device__ __forceinline__ void store(double* p) const { *reinterpret_cast<float2*>(p) = make_float2(hi, lo); }
  // (hi, lo) - d: two-sum of hi and -d, then renormalise (fast two-sum)
  __device__ __forceinline__ void sub(float d) {
    const float s = hi - d;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (-d - bb);
    const float l = lo + e;
    const float h = s + l;
    lo = l - (h - s);
    hi = h;
  }
  __device__ __forceinline__ bool used_up() const {
    const int h = __float_as_int(hi);
    return h < 0 || (h == 0 && __float_as_int(lo) <= 0);
  }
  __device__ __forceinline__ bool dead() const { return __float_as_int(hi) == 0x7f800000; }
  static __device__ __forceinline__ Tau fresh(float x) { return Tau{x, 0.0f}; }
  static __device__ __forceinline__ Tau infinite() { return Tau{__int_as_float(0x7f800000), 0.0f}; }
  static __device__ __forceinline__ Tau one() { return Tau{1.0f, 0.0f}; }
};

// Conversions between the double tau of the C ABI and the stored representation.
template <typename R> __device__ __forceinline__ void store_tau_from_double(double* p, double t);
template <> __device__ __forceinline__ void store_tau_from_double<double>(double* p, double t) { *p = t; }
template <> __device__ __forceinline__ void store_tau_from_double<float>(double* p, double t) {
  const float hi = (float)t;
  const float lo = isinf(t) ? 0.0f : (float)(t - (double)hi);
  Tau<float>{hi, lo}.store(p);
}
template <typename R> __device__ __forceinline__ double tau_to_double(const double* p);
template <> __device__ __forceinline__ double tau_to_double<double>(const double* p) { return *p; }
template <> __device__ __forceinline__ double tau_to_double<float>(const double* p) {
  const Tau<float> t = Tau<float>::load(p);
  return (double)t.hi + (double)t.lo;
}

// Uniform draws in the working precision.  FP64: U = (m + 1/2) 2^-52 (m the top 52 bits of the
// word) as in the oracle.  FP32: the correctly rounded float of that same U, and of 1 - U, from
// the 53-bit odd integers 2m + 1 and 2^53 - 1 - 2m (integer-to-float conversion, no FP64).
template <typename R> struct Uniform;
template <> struct Uniform<double> {
  double u, v;
  static __device__ __forceinline__ Uniform from(uint64_t w) {
    const double u = u01(w);
    return Uniform{u, 1.0 - u};
  }
};
template <> struct Uniform<float> {
  float u, v;
  static __device__ __forceinline__ Uniform from(uint64_t w) {
    const unsigned long long m = w >> 12;
    return Uniform{__ull2float_rn(2ull * m + 1ull) * 0x1.0p-53f,
                   __ull2float_rn((1ull << 53) - 1ull - 2ull * m) * 0x1.0p-53f};
  }
};

template <typename R>
__device__ __forceinline__ void draw4r(uint64_t seed, uint64_t scen, uint64_t id, uint64_t step, uint64_t kind,
                                       uint64_t purpose, Uniform<R> U[4]) {
  uint64_t c[4] = {id, step, kind, purpose};
  philox4x64(c, seed, scen);
#pragma unroll
  for (int i = 0; i < 4; ++i) U[i] = Uniform<R>::from(c[i]);
}

}  // namespace qedlib
