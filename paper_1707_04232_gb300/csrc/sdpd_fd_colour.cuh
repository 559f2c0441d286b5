// sdpd_fd_colour.cuh -- one pair update of the fluctuation/dissipation sweep
// (Sections 3.2-3.3) and the colour kernel that runs a colour's blocks level
// by level.  Included by one translation unit per precision, each of which
// instantiates the block-schedule variants of its precision.
#pragma once
#include <algorithm>
#include <type_traits>

#include "sdpd_fd_common.cuh"

namespace sdpd {

// ---------------------------------------------------------------------------
// One pair update.
// ---------------------------------------------------------------------------
template <class R>
struct FDConst {
  R m, inv_m, half_m, inv_h, cF;
  R kpar_m2, kperp_m2;  // (10/3 eta + 4 zeta) m^2, (5/3 eta - zeta) m^2
  R inv_C_K, kB, two_over_CK, dt_over_m;
  R CKm1;               // C_K / kB - 1
  R four_kB_over_m;
  double CKm1_d;          // C_K / kB - 1 in float64 (the exact Metropolis ratio)
  float nq_hi, nq_lo;     // -1 / (4 m) as a float-float (energy change from momenta)
  int scheme;
};

// Elementary functions of the sweep.  float64: the correctly rounded /
// accurate library versions.  float32 (mixed path): hardware approximations
// (relative error ~1e-7) for the proposal coefficients and Box-Muller -- the
// Metropolis step stays exact for any deterministic proposal coefficients
// because the forward and reverse moves use the same functions -- and the
// accurate log1p for the entropy term of the target measure.
namespace fm {
__device__ __forceinline__ double div(double a, double b) { return a / b; }
__device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double exp(double x) { return ::exp(x); }
__device__ __forceinline__ float exp(float x) { return __expf(x); }
__device__ __forceinline__ double log(double x) { return ::log(x); }
__device__ __forceinline__ float log(float x) { return __logf(x); }
__device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
__device__ __forceinline__ float sqrt(float x) { return x * rsqrtf(x); }
__device__ __forceinline__ double rsqrt(double x) { return x > 1e-30 ? pair_rinv(x) : 1.0 / ::sqrt(x); }
__device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double expm1(double x) { return ::expm1(x); }
// exp(x) - 1 for x <= 0: Taylor polynomial for small |x| (relative error
// < 1e-8 below 1/8), the hardware exponential above
__device__ __forceinline__ float expm1(float x) {
  if (x > -0.125f) return x * (1.0f + x * (0.5f + x * (1.0f / 6.0f + x * (1.0f / 24.0f + x * (1.0f / 120.0f + x * (1.0f / 720.0f))))));
  return __expf(x) - 1.0f;
}
__device__ __forceinline__ double log1p(double x) { return ::log1p(x); }
// log(1 + x): alternating series for |x| < 1/16 (relative error < 2e-8),
// the hardware logarithm of 1 + x above
__device__ __forceinline__ float log1p(float x) {
  if (fabsf(x) < 0.0625f)
    return x * (1.0f - x * (0.5f - x * (1.0f / 3.0f - x * (0.25f - x * (0.2f - x * (1.0f / 6.0f))))));
  return __logf(1.0f + x);
}
}  // namespace fm

// Error-free transformations in float32 (Knuth's two-sum, the FMA split of
// a product): a + b = s + e and a * b = p + e exactly.  The rounded
// intrinsics keep the compiler from contracting or reordering them.
namespace eft {
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
}  // namespace eft

// Box-Muller normals and the uniform of one pair at one sweep (see
// pair_randoms), float32 path: the float64 path's uniforms rounded to
// float32 with full relative precision (a fixed-point uniform would lose
// the relative precision of the small values that the logarithms of
// Box-Muller and of the Metropolis test magnify), the logarithm inside
// Box-Muller accurate near 1 (log1p of minus 1 - u, formed from the
// integer), angles reduced to [-pi, pi) for the hardware sine and cosine.
__device__ __forceinline__ float uniform53f(uint64_t w) {  // (top 53 bits + 1/2) 2^-53
  const uint64_t m = w >> 11;
  const float hi = (float)(uint32_t)(m >> 21), lo = (float)(uint32_t)(m & 0x1fffffull) + 0.5f;
  return __fmaf_rn(hi, 2.3283064365386963e-10f, lo * 1.1102230246251565e-16f);
}
__device__ __forceinline__ float uniform32f(uint32_t x) {  // (x + 1/2) 2^-32
  return ((float)x + 0.5f) * 2.3283064365386963e-10f;
}
// -2 ln u for the radius of Box-Muller.  Below 1/2 the logarithm of u
// itself; above, log1p(-(1 - u)) with 1 - u = (c + 1/2) 2^-b formed from the
// integer complement c = 2^b - 1 - m, because u rounded to float32 reaches
// 1 for the largest m (and -2 ln u would then be 0 instead of ~2^-b).
__device__ __forceinline__ float neg2log_u53(uint64_t w) {  // u = (top 53 bits m + 1/2) 2^-53
  const uint64_t m = w >> 11;
  if (m < (1ull << 52)) return -2.0f * __logf(uniform53f(w));
  const uint64_t c = ((1ull << 53) - 1ull) - m;
  const float t = __fmaf_rn((float)(uint32_t)(c >> 21), 2.3283064365386963e-10f,
                            ((float)(uint32_t)(c & 0x1fffffull) + 0.5f) * 1.1102230246251565e-16f);
  return -2.0f * fm::log1p(-t);
}
__device__ __forceinline__ float neg2log_u32(uint32_t x) {  // u = (x + 1/2) 2^-32
  if (x < 0x80000000u) return -2.0f * __logf(uniform32f(x));
  return -2.0f * fm::log1p(-(((float)(0xffffffffu - x) + 0.5f) * 2.3283064365386963e-10f));
}
__device__ __forceinline__ void pair_randoms_fast(uint64_t seed, uint64_t sweep, uint64_t idi, uint64_t idj,
                                                  float G[3], float* U) {
  uint64_t w[4];
  philox4x64_10(sweep, idi, idj, 0ull, seed, 0ull, w);
  const float twopi = 6.28318530717958647692f;
  const float u1 = uniform53f(w[1]);
  const float R = fm::sqrt(neg2log_u53(w[0]));
  float sn, cs;
  __sincosf(twopi * (u1 - 0.5f), &sn, &cs);  // the angle 2 pi u1 - pi
  G[0] = -R * cs;
  G[1] = -R * sn;
  const float u3 = uniform32f((uint32_t)(w[2] & 0xffffffffull));
  G[2] = -fm::sqrt(neg2log_u32((uint32_t)(w[2] >> 32))) * __cosf(twopi * (u3 - 0.5f));
  *U = uniform53f(w[3]);
}
__device__ __forceinline__ void pair_randoms_fast(uint64_t seed, uint64_t sweep, uint64_t idi, uint64_t idj,
                                                  double G[3], double* U) {
  pair_randoms(seed, sweep, idi, idj, G, U);
}

// alpha = exp(-2 gamma dt / m) and zt = (2/m) zeta of Section 3.2 for both
// directions at energies (ei, ej), with gamma = kappa (1 - d) and
// sigma = 2 sqrt(kappa kB Ti Tj / (Ti + Tj)) of Eq. (sdpd-gamma-sigma):
// zt^2 = sigma^2 (1 - alpha^2) / (m gamma) = 4 kB Ti Tj / ((Ti+Tj) m (1-d)) (1 - alpha^2)
// (kappa cancels).  Ideal gas: T = eps / C_K and C = C_K, so
// d = kB Ti Tj / (Ti + Tj)^2 * 2 / C_K.
//
// Returns m = alpha - 1 = expm1(x) per direction (alpha itself is 1 + m):
// one expm1 per direction gives both alpha and 1 - alpha^2 = -m (2 + m), and
// one reciprocal of Ti + Tj serves both quotients -- the float64 dependency
// chain of a pair update is what bounds the sweep when a colour has few
// blocks.
template <class R>
__device__ __forceinline__ void pair_coeffs(const FDConst<R>& k, R kpar, R kperp, R ei, R ej, R& mpar,
                                            R& mperp, R& zpar, R& zperp) {
  const R Ti = ei * k.inv_C_K, Tj = ej * k.inv_C_K;
  const R isT = fm::div(R(1), Ti + Tj);
  const R hT = Ti * Tj * isT;
  const R omd = R(1) - k.kB * k.two_over_CK * hT * isT;
  const R xpar = R(-2) * kpar * omd * k.dt_over_m;  // log alpha per direction
  const R xperp = R(-2) * kperp * omd * k.dt_over_m;
  mpar = fm::expm1(xpar);
  mperp = fm::expm1(xperp);
  const R s = fm::div(k.four_kB_over_m * hT, omd);
  zpar = fm::sqrt(s * (-mpar * (R(2) + mpar)));
  zperp = fm::sqrt(s * (-mperp * (R(2) + mperp)));
}

// State-dependent part of one float64 pair update on (p_i, p_j) with
// internal energies (ei, ej), given the pair's unit vector e = r_ij / r_ij,
// base = F(r_ij) / (rho_i rho_j), its Gaussians G and the logarithm lnU of its
// uniform.  Returns 0 accept, 1 energy-bound reject, 2 Metropolis reject;
// deps receives the energy change shared by the two particles (applied by the
// caller on acceptance).
__device__ __forceinline__ int fd_pair(const FDConst<double>& k, double ex, double ey, double ez, double base,
                                       const double G[3], double lnU, double* pi, double* pj, double ei,
                                       double ej, double& deps, double& margin, bool& negative) {
  using R = double;
  const R kpar = k.kpar_m2 * base, kperp = k.kperp_m2 * base;
  margin = R(0);
  deps = R(0);
  if (!(kperp > R(0)) || !(kpar > R(0))) return 0;  // at r = h the pair does nothing
  const R vx = (pi[0] - pj[0]) * k.inv_m, vy = (pi[1] - pj[1]) * k.inv_m, vz = (pi[2] - pj[2]) * k.inv_m;
  R mpar, mperp, zpar, zperp;
  pair_coeffs(k, kpar, kperp, ei, ej, mpar, mperp, zpar, zperp);
  const R apar = R(1) + mpar, aperp = R(1) + mperp;
  // proposal, Eq. (proposal): v' = sum_theta P^theta (alpha^theta v + zt^theta G)
  const R vpar = ex * vx + ey * vy + ez * vz;
  const R gpar = ex * G[0] + ey * G[1] + ez * G[2];
  const R cpar = (apar - aperp) * vpar + (zpar - zperp) * gpar;
  const R wx = aperp * vx + zperp * G[0] + cpar * ex;
  const R wy = aperp * vy + zperp * G[1] + cpar * ey;
  const R wz = aperp * vz + zperp * G[2] + cpar * ez;
  // momenta of Eq. (proposal-update), energy shared equally (Section 3.2)
  const R dpx = k.half_m * (wx - vx), dpy = k.half_m * (wy - vy), dpz = k.half_m * (wz - vz);
  const R nix = pi[0] + dpx, niy = pi[1] + dpy, niz = pi[2] + dpz;
  const R njx = pj[0] - dpx, njy = pj[1] - dpy, njz = pj[2] - dpz;
  const double ko = pi[0] * pi[0] + pj[0] * pj[0] + pi[1] * pi[1] + pj[1] * pj[1] + pi[2] * pi[2] + pj[2] * pj[2];
  const double kn = nix * nix + njx * njx + niy * niy + njy * njy + niz * niz + njz * njz;
  deps = -0.5 * (kn - ko) * (0.5 * k.inv_m);
  // energy bound, Eq. (energy-bound): both new internal energies > 0
  const R emin = (ei < ej ? ei : ej) + deps;
  margin = emin;
  int decision = 0;
  if (k.scheme == SDPD_SCHEME_SSA) {
    if (!(emin > R(0))) negative = true;
  } else if (!(emin > R(0))) {
    decision = 1;
  } else if (k.scheme == SDPD_SCHEME_EMS) {
    // Metropolis ratio, Eq. (metropolis-ratio): the reverse move from v'
    // with the coefficients at the proposed energies
    R mrpar, mrperp, ypar, yperp;
    pair_coeffs(k, kpar, kperp, ei + deps, ej + deps, mrpar, mrperp, ypar, yperp);
    const R bpar = R(1) + mrpar, bperp = R(1) + mrperp;
    // one reciprocal for both directions of the reverse move's noise scale
    const R ryy = fm::div(R(1), ypar * yperp);
    const R ipar = yperp * ryy, ip = ypar * ryy;  // 1 / zt'_par, 1 / zt'_perp
    // reverse noise B'^-1 (v - A' v') from the proposed v' itself
    const R wpar = ex * wx + ey * wy + ez * wz;
    const R cb = (bpar - bperp) * wpar;
    const R bx = vx - (bperp * wx + cb * ex), by = vy - (bperp * wy + cb * ey), bz = vz - (bperp * wz + cb * ez);
    const R spar = ex * bx + ey * by + ez * bz;
    const R cq = (ipar - ip) * spar;
    const R qx = bx * ip + cq * ex, qy = by * ip + cq * ey, qz = bz * ip + cq * ez;
    const R quad = qx * qx + qy * qy + qz * qz;
    const R g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    // log|B(v)| - log|B(v')| with |B| = zt_par zt_perp^2
    const R ldet = fm::log(zpar * zperp * zperp * (ipar * ip * ip));
    // (S(eps') - S(eps))/kB - (log T(eps') - log T(eps)) = (C_K/kB - 1) log(eps'/eps)
    // summed over the two particles: log1p(x) + log1p(y) = log1p(x + y + x y)
    // with x = deps/ei, y = deps/ej, i.e. deps (ei + ej + deps) / (ei ej)
    const R ent = k.CKm1 * fm::log1p(fm::div(deps * (ei + ej + deps), ei * ej));
    const R a = R(0.5) * (g2 - quad) + ldet + ent;
    const R mg = a - lnU;
    margin = mg;
    if (mg < R(0)) decision = 2;  // U > exp(a)
  }
  if (decision == 0) {
    pi[0] = nix; pi[1] = niy; pi[2] = niz;
    pj[0] = njx; pj[1] = njy; pj[2] = njz;
  }
  return decision;
}

// The float32 quantities that define a mixed-path proposal and its reverse
// move, with the float64 energies: everything the Metropolis log-ratio of
// Eq. (metropolis-ratio) is evaluated from.  alpha = 1 + m per direction
// (m = expm1 of the exponent, so alpha - 1 carries no rounding of its own),
// zt the noise scales; the r-suffixed values belong to the reverse move at
// the proposed energies.
struct MixedRatioIn {
  float ex, ey, ez, vx, vy, vz, g0, g1, g2, u;
  float mpar, mperp, zpar, zperp, mrpar, mrperp, ypar, yperp;
  double ei, ej, deps;
};

// The Metropolis margin a - ln U of a mixed-path pair evaluated in float64
// from its float32 inputs: the reference value that the float32 evaluation
// approximates.  Reverse noise per direction theta,
// G'_theta = [(1 - alpha'_theta alpha_theta) v_theta - alpha'_theta zt_theta G_theta] / zt'_theta,
// which is B'^-1 (v - A' v') for v' = A v + B G; a = (|G|^2 - |G'|^2)/2 +
// log(|B| / |B'|) + (C_K/kB - 1) log1p(deps (ei + ej + deps) / (ei ej)).
// Kept out of line: it runs only for the rare pairs whose float32 margin is
// within its error bound of zero (and for every pair when records are kept).
static __device__ __noinline__ double mixed_margin_fp64(const MixedRatioIn& r, double CKm1) {
  const double ex = r.ex, ey = r.ey, ez = r.ez, vx = r.vx, vy = r.vy, vz = r.vz;
  const double g0 = r.g0, g1 = r.g1, g2 = r.g2;
  const double mpar = r.mpar, mperp = r.mperp, mrpar = r.mrpar, mrperp = r.mrperp;
  const double zpar = r.zpar, zperp = r.zperp, ypar = r.ypar, yperp = r.yperp;
  const double vpar = ex * vx + ey * vy + ez * vz;
  const double gpar = ex * g0 + ey * g1 + ez * g2;
  const double cpar = -(mpar + mrpar + mpar * mrpar), cperp = -(mperp + mrperp + mperp * mrperp);
  const double bpar = (1.0 + mrpar) * zpar, bperp = (1.0 + mrperp) * zperp;
  const double qpar = (cpar * vpar - bpar * gpar) / ypar;
  const double qx = (cperp * (vx - vpar * ex) - bperp * (g0 - gpar * ex)) / yperp;
  const double qy = (cperp * (vy - vpar * ey) - bperp * (g1 - gpar * ey)) / yperp;
  const double qz = (cperp * (vz - vpar * ez) - bperp * (g2 - gpar * ez)) / yperp;
  const double quad = qpar * qpar + qx * qx + qy * qy + qz * qz;
  const double gg = g0 * g0 + g1 * g1 + g2 * g2;
  const double ldet = log((zpar * zperp * zperp) / (ypar * yperp * yperp));
  const double ent = CKm1 * log1p(r.deps * (r.ei + r.ej + r.deps) / (r.ei * r.ej));
  return 0.5 * (gg - quad) + ldet + ent - log((double)r.u);
}

// One pair update of the mixed path.  The pair arithmetic (geometry,
// coefficients, proposal, momenta) is float32.  The internal energies are
// float64 in the state; during a block visit a particle's energy is its
// float64 value at load plus the visit's changes, which are kept as a
// float-float sum (about 48 significant bits).  The energy change deps of a
// pair is computed exactly from the float32 momenta before and after the
// move: -1/(4m) sum (new^2 - old^2), each square split exactly by an FMA and
// the differences and sums carried by two-sum, to float-float accuracy
// (dh + dl).  This keeps every pair update energy-conserving to float64
// rounding without float64 instructions, of which GB300 issues one for
// every 64 float32 ones.
//
// The energy bound is decided in float32 when its margin is clearly away
// from zero, else in float64 from the exact energies.  The Metropolis test
// is decided in float64: the log-ratio is evaluated in float32 together with
// a bound on its rounding error (a running error analysis of every
// operation, the documented error of the hardware logarithm, and a factor 2
// of safety), and a pair whose float32 margin is within that bound of zero
// is re-evaluated by mixed_margin_fp64, so every decision is the one the
// float64 evaluation of the same ratio gives.  m32 and tol receive the
// float32 margin and its bound; margin the float64 margin whenever it was
// evaluated (always when `exact` is set).  exact_e(ei, ej) gives the two
// current energies in float64 and uniform() the pair's uniform U (both for
// the rare float64 evaluations).
template <class ExactE, class Uniform>
__device__ __forceinline__ int fd_pair_mixed(const FDConst<float>& k, float ex, float ey, float ez, float base,
                                             const float G[3], Uniform uniform, float lnU, float* pi, float* pj,
                                             float eif, float ejf, ExactE exact_e, float& dh, float& dl,
                                             double& margin, float& m32, float& tol, bool exact,
                                             bool& negative) {
  const float kpar = k.kpar_m2 * base, kperp = k.kperp_m2 * base;
  margin = 0.0;
  dh = 0.0f;
  dl = 0.0f;
  m32 = 0.0f;
  tol = 0.0f;
  if (!(kperp > 0.0f) || !(kpar > 0.0f)) return 0;  // at r = h the pair does nothing
  const float vx = (pi[0] - pj[0]) * k.inv_m, vy = (pi[1] - pj[1]) * k.inv_m, vz = (pi[2] - pj[2]) * k.inv_m;
  float mpar, mperp, zpar, zperp;  // alpha - 1 and zt per direction
  pair_coeffs(k, kpar, kperp, eif, ejf, mpar, mperp, zpar, zperp);
  // proposal, Eq. (proposal), as the velocity change
  // v' - v = m_perp v + zt_perp G + [(m_par - m_perp) v_par + (zt_par - zt_perp) G_par] e
  const float vpar = ex * vx + ey * vy + ez * vz;
  const float gpar = ex * G[0] + ey * G[1] + ez * G[2];
  const float cpar = (mpar - mperp) * vpar + (zpar - zperp) * gpar;
  const float dvx = mperp * vx + zperp * G[0] + cpar * ex;
  const float dvy = mperp * vy + zperp * G[1] + cpar * ey;
  const float dvz = mperp * vz + zperp * G[2] + cpar * ez;
  // momenta of Eq. (proposal-update), energy shared equally (Section 3.2)
  const float dpx = k.half_m * dvx, dpy = k.half_m * dvy, dpz = k.half_m * dvz;
  const float nn[6] = {pi[0] + dpx, pi[1] + dpy, pi[2] + dpz, pj[0] - dpx, pj[1] - dpy, pj[2] - dpz};
  // float32 estimate of the energy change: it places the reverse move's
  // coefficients (at eps + deps, rounded to float32, where it agrees with the
  // exact value below to a float32 rounding) without waiting for the exact
  // float-float sum, which takes a longer dependency chain
  float dhf;
  {
    float dk = 0.0f;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      dk = fmaf(nn[t] - pi[t], nn[t] + pi[t], dk);
      dk = fmaf(nn[t + 3] - pj[t], nn[t + 3] + pj[t], dk);
    }
    dhf = k.nq_hi * dk;
  }
  {  // deps = -1/2 of the kinetic-energy change of the stored momenta, exactly
    const float oo[6] = {pi[0], pi[1], pi[2], pj[0], pj[1], pj[2]};
    float d[6], lo[6];  // new^2 - old^2 per component as d + lo, exactly
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      float pn, en, po, eo, ed;
      eft::two_prod(nn[t], nn[t], pn, en);
      eft::two_prod(oo[t], oo[t], po, eo);
      eft::two_sum(pn, -po, d[t], ed);
      lo[t] = __fadd_rn(ed, __fsub_rn(en, eo));
    }
    // the six high parts summed by a tree of two-sums (depth 3), the low
    // parts and the two-sum errors plainly (they are 2^-24 of the result)
    float s01, e01, s23, e23, s45, e45, s03, e03, Dh, eD, Dl;
    eft::two_sum(d[0], d[1], s01, e01);
    eft::two_sum(d[2], d[3], s23, e23);
    eft::two_sum(d[4], d[5], s45, e45);
    eft::two_sum(s01, s23, s03, e03);
    eft::two_sum(s03, s45, Dh, eD);
    Dl = __fadd_rn(__fadd_rn(__fadd_rn(lo[0], lo[1]), __fadd_rn(lo[2], lo[3])),
                   __fadd_rn(__fadd_rn(lo[4], lo[5]), __fadd_rn(__fadd_rn(e01, e23), __fadd_rn(e45, __fadd_rn(e03, eD)))));
    eft::two_sum(Dh, Dl, Dh, Dl);  // renormalise
    // times -1/(4m) (a float-float constant)
    float ph, pl;
    eft::two_prod(Dh, k.nq_hi, ph, pl);
    pl = __fmaf_rn(Dh, k.nq_lo, __fmaf_rn(Dl, k.nq_hi, pl));
    eft::two_sum(ph, pl, dh, dl);
  }
  // energy bound, Eq. (energy-bound): both new internal energies > 0;
  // float32 decides unless the margin is within its rounding of zero
  const float eminf = eif < ejf ? eif : ejf;
  float emn = eminf + dh;
  if (fabsf(emn) <= 32.0f * 5.9604645e-8f * (eminf + fabsf(dh))) {
    double ei, ej;
    exact_e(ei, ej);
    emn = ((ei < ej ? ei : ej) + ((double)dh + (double)dl)) > 0.0 ? 1.0f : -1.0f;
  }
  if (exact) margin = (double)emn;  // (float64 work only where it is asked for)
  int decision = 0;
  if (k.scheme == SDPD_SCHEME_SSA) {
    if (!(emn > 0.0f)) negative = true;
  } else if (!(emn > 0.0f)) {
    decision = 1;
  } else if (k.scheme == SDPD_SCHEME_EMS) {
    // reverse move from v' with the coefficients at the proposed energies
    float mrpar, mrperp, ypar, yperp;
    pair_coeffs(k, kpar, kperp, eif + dhf, ejf + dhf, mrpar, mrperp, ypar, yperp);
    // 1 - alpha' alpha = -(m + m' + m m') (both m <= 0: no cancellation), alpha' zt
    const float cpr = -(mpar + mrpar + mpar * mrpar), cqr = -(mperp + mrperp + mperp * mrperp);
    const float bzpar = fmaf(mrpar, zpar, zpar), bzperp = fmaf(mrperp, zperp, zperp);
    const float ryy = fm::div(1.0f, ypar * yperp);
    const float ipar = yperp * ryy, ip = ypar * ryy;  // 1 / zt'_par, 1 / zt'_perp
    // reverse noise B'^-1 (v - A' v') = B'^-1 [(I - A' A) v - A' B G] per
    // direction: no cancellation when zt' -> 0 (pairs near the cut-off)
    const float qpar = (cpr * vpar - bzpar * gpar) * ipar;
    const float qx = (cqr * (vx - vpar * ex) - bzperp * (G[0] - gpar * ex)) * ip;
    const float qy = (cqr * (vy - vpar * ey) - bzperp * (G[1] - gpar * ey)) * ip;
    const float qz = (cqr * (vz - vpar * ez) - bzperp * (G[2] - gpar * ez)) * ip;
    const float quad = qpar * qpar + qx * qx + qy * qy + qz * qz;
    const float g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    // log|B(v)| - log|B(v')| with |B| = zt_par zt_perp^2
    const float ldet = fm::log(zpar * zperp * zperp * (ipar * ip * ip));
    // (S(eps') - S(eps))/kB - (log T(eps') - log T(eps)) over both particles
    const float x = fm::div(dh * (eif + ejf + dh), eif * ejf);
    const float ent = k.CKm1 * fm::log1p(x);
    const float mg = 0.5f * (g2 - quad) + ldet + ent - lnU;
    // error bound of mg against its exact value for these inputs (u = 2^-24;
    // 3.6e-7 bounds the absolute error of the hardware logarithm on
    // [0.5, 2], 3 ulp elsewhere)
    const float u = 5.9604645e-8f, elog = 3.6e-7f;
    const float V = fabsf(vx) + fabsf(vy) + fabsf(vz), Gs = fabsf(G[0]) + fabsf(G[1]) + fabsf(G[2]);
    const float qm = fabsf(qpar) * ipar * (fabsf(cpr) * V + bzpar * Gs) +
                     (fabsf(qx) + fabsf(qy) + fabsf(qz)) * ip * (fabsf(cqr) * V + bzperp * Gs);
    const float T = 8.0f * g2 + 23.0f * quad + 32.0f * qm + 11.0f * fabsf(ldet) + 25.0f * fabsf(ent) +
                    11.0f * fabsf(lnU) + 23.0f;
    tol = 2.0f * (u * T + 2.0f * elog);
    if (fabsf(x) >= 0.0625f) tol += 2.0f * k.CKm1 * (elog + 16.0f * u);
    m32 = mg;
    if (exact || !(fabsf(mg) > tol)) {  // float32 not decisive (or NaN): float64
      MixedRatioIn r;
      r.ex = ex; r.ey = ey; r.ez = ez; r.vx = vx; r.vy = vy; r.vz = vz;
      r.g0 = G[0]; r.g1 = G[1]; r.g2 = G[2]; r.u = uniform();
      r.mpar = mpar; r.mperp = mperp; r.zpar = zpar; r.zperp = zperp;
      r.mrpar = mrpar; r.mrperp = mrperp; r.ypar = ypar; r.yperp = yperp;
      exact_e(r.ei, r.ej);
      r.deps = (double)dh + (double)dl;
      margin = mixed_margin_fp64(r, k.CKm1_d);
      if (margin < 0.0) decision = 2;  // U > exp(a)
    } else if (mg < 0.0f) {  // decided in float32: |mg| exceeds its error bound
      decision = 2;
    }
  }
  if (decision == 0) {
    pi[0] = nn[0]; pi[1] = nn[1]; pi[2] = nn[2];
    pj[0] = nn[3]; pj[1] = nn[4]; pj[2] = nn[5];
  }
  return decision;
}

// ---------------------------------------------------------------------------
// One colour of the sweep.  A warp runs OPW blocks of the colour
// side by side, each on its own group of lanes, in lockstep over the blocks'
// dependency levels.
//
// A block's particles (momenta and energies) live in shared memory.  The
// block's pairs are consumed in chunks of kChunk consecutive pairs of its
// level-ordered list: first every lane of the group stages the chunk's
// state-independent data (unit vector, F(r)/(rho_i rho_j), random numbers),
// then the chunk's levels (or parts of a level: pairs of one level are
// independent) run one after the other, the lanes of the group sharing a
// level's pairs.
// ---------------------------------------------------------------------------
constexpr int kChunk = 32;

// Cell code inside the block of owner (ox, oy, oz) of a particle whose cell
// bits are w: bit k set iff the particle sits in the upper cell along axis k.
template <class T>
__device__ __forceinline__ int block_code(T w, int ox, int oy, int oz) {
  int cx, cy, cz;
  unpack_cell(w_to_cellbits(w), cx, cy, cz);
  return (cx != ox) | ((cy != oy) << 1) | ((cz != oz) << 2);
}

template <class R>
struct FdSmemBase {
  R px[kMaxBlock], py[kMaxBlock], pz[kMaxBlock];
  int32_t cst[8], cbs[8];  // the block's cells: first storage index, offset in the block
  // staged pair data of the current chunk
  R G0[kChunk], G1[kChunk], G2[kChunk], lnU[kChunk];
  R ex[kChunk], ey[kChunk], ez[kChunk], base[kChunk];
  uint16_t pr[kChunk];
  uint16_t off[kMaxLevels + 1];  // level offsets of the block's pair list
};
template <class R>
struct FdSmem;
// float64 pair arithmetic: the energies themselves
template <>
struct FdSmem<double> : FdSmemBase<double> {
  double e[kMaxBlock];
};
// float32 pair arithmetic: each particle's energy as a running float32 sum
// es (the energy at load rounded to float32, plus the visit's changes) and
// its compensation ec (the rounding errors of that sum and the low parts of
// the changes), so that the energy is eps(load) + (es - (float)eps(load)) + ec
template <>
struct FdSmem<float> : FdSmemBase<float> {
  float es[kMaxBlock], ec[kMaxBlock];
};

// A block beyond the capacities of the shared-memory schedule (kHdrBig: more
// than kMaxBlock particles, kMaxPairs owned pairs or kMaxLevels levels).
// The whole warp sweeps its owned pairs in canonical order, one pair after
// the other, on the state in global memory; slow, but any block completes
// with the result of the sequential sweep.  The block's particles in rank
// order (ids ascending) go to its place in big_perm (blocks of one colour
// are disjoint, so N entries suffice).  Row d of
// the canonical order holds the pairs (perm[r], perm[r + d]), r ascending;
// the lanes test 32 candidates of a row at once (owner rule, then the
// neighbour predicate of the schedule enumeration) and lane 0 updates the
// hits in order of r.
// pair counters and flags of a sequential block sweep
struct BigCounts {
  unsigned long long tot, acc, rb, rm;
  int negative, bad;
};

template <class P, class A, int KIND>
__device__ __noinline__ BigCounts fd_big_block(const Consts& c, const FDConst<typename A::R>& k, const Arrays<P>& a,
                                          typename P::V4* __restrict__ qp4, const int32_t* __restrict__ cell_start,
                                          const int32_t* __restrict__ mrank, const uint32_t* xmx,
                                          const uint32_t* xmy, const uint32_t* xmz, int64_t o, int ox, int oy,
                                          int oz, int colour, uint64_t seed, uint64_t sweep, sdpd_pair_rec* recs,
                                          unsigned long long* rec_count, int64_t rec_cap, int32_t* perm) {
  using R = typename A::R;
  using S = typename P::R;
  using V4 = typename P::V4;
  constexpr bool kSame = std::is_same<R, S>::value;
  const int lane = threadIdx.x & 31;
  unsigned long long n_tot = 0, n_acc = 0, n_rb = 0, n_rm = 0;
  bool negative = false, bad = false;
  BlockCells b;
  block_cells(c, ox, oy, oz, mrank, cell_start, b);
  const int nb = b.base[8];
  for (int q = lane; q < nb; q += 32) {  // rank order: every cell holds its ids ascending
    const int d = cell_code_of(b, q);
    const int g = b.start[d] + (q - b.base[d]);
    const int32_t id = a.id[g];
    int r = 0;
    for (int e = 0; e < 8; ++e) {  // ids of cell e below id
      int lo = b.start[e], n = b.cnt[e];
      while (n > 0) {
        const int half = n >> 1;
        if (a.id[lo + half] < id) { lo += half + 1; n -= half + 1; }
        else n = half;
      }
      r += lo - b.start[e];
    }
    perm[r] = g;
  }
  __syncwarp();
  BlockGeom<P> geo;
  geo.init(c, ox, oy, oz, xmx, xmy, xmz);
  const S h2 = (S)c.h2, inv_h = (S)(1.0 / c.h), cF = (S)c.cF;
  int seq = 0;
  for (int d = 1; d < nb; ++d) {
    for (int r0 = 0; r0 < nb - d; r0 += 32) {
      const int r = r0 + lane;
      int gA = 0, gB = 0;
      bool hit = false;
      if (r < nb - d) {
        gA = perm[r];
        gB = perm[r + d];
        const V4 qa = ld4(&a.q4[gA]), qb = ld4(&a.q4[gB]);
        const int dA = block_code(qa.w, ox, oy, oz), dB = block_code(qb.w, ox, oy, oz);
        const int hb = (int)owner_bits(a.id[gA]);
        if ((((dA ^ hb) & ~(dA ^ dB)) & 7) == 0) {  // owned: on shared axes the cell bit equals the owner bit
          S xa, ya, za, xb, yb, zb, rx, ry, rz;
          geo.local(qa, dA, xa, ya, za);
          geo.local(qb, dB, xb, yb, zb);
          geo.disp(xa, ya, za, xb, yb, zb, rx, ry, rz);
          hit = r2_of(rx, ry, rz) < h2;
        }
      }
      unsigned m = __ballot_sync(0xffffffffu, hit);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int ga = __shfl_sync(0xffffffffu, gA, src), gb = __shfl_sync(0xffffffffu, gB, src);
        if (lane == 0) {
          const V4 qa = ld4(&a.q4[ga]), qb = ld4(&a.q4[gb]);
          S xa, ya, za, xb, yb, zb, rx, ry, rz;
          geo.local(qa, block_code(qa.w, ox, oy, oz), xa, ya, za);
          geo.local(qb, block_code(qb.w, ox, oy, oz), xb, yb, zb);
          geo.disp(xa, ya, za, xb, yb, zb, rx, ry, rz);
          const S r2 = r2_of(rx, ry, rz);
          const S inv_r = fm::rsqrt(r2);
          const R ex = (R)(rx * inv_r), ey = (R)(ry * inv_r), ez = (R)(rz * inv_r);
          const R bs = (R)fm::div(kernel_F<KIND>(r2 * inv_r * inv_h, cF), a.rho[ga] * a.rho[gb]);
          R G[3], U;
          pair_randoms_fast(seed, sweep, (uint64_t)a.id[ga], (uint64_t)a.id[gb], G, &U);
          const R lnU = k.scheme == SDPD_SCHEME_EMS ? fm::log(U) : U;
          R pa[3] = {(R)a.px[ga], (R)a.py[ga], (R)a.pz[ga]};
          R pb[3] = {(R)a.px[gb], (R)a.py[gb], (R)a.pz[gb]};
          const R pa0[3] = {pa[0], pa[1], pa[2]}, pb0[3] = {pb[0], pb[1], pb[2]};
          double margin;
          float m32 = 0.0f, tol = 0.0f;
          int dcs;
          if constexpr (A::mixed) {
            auto exact_e = [&](double& x, double& y) { x = a.eps[ga]; y = a.eps[gb]; };
            float dh, dl;
            auto uniform = [&]() { return U; };
            dcs = fd_pair_mixed(k, ex, ey, ez, bs, G, uniform, lnU, pa, pb, (float)a.eps[ga], (float)a.eps[gb],
                                exact_e, dh, dl, margin, m32, tol, recs != nullptr, negative);
            if (dcs == 0) {
              const double de = (double)dh + (double)dl;
              a.eps[ga] += de;
              a.eps[gb] += de;
            }
          } else {
            double deps;
            dcs = fd_pair(k, ex, ey, ez, bs, G, lnU, pa, pb, a.eps[ga], a.eps[gb], deps, margin, negative);
            if (dcs == 0) {
              a.eps[ga] = a.eps[ga] + deps;
              a.eps[gb] = a.eps[gb] + deps;
            }
          }
          if (dcs == 0) {
            if constexpr (kSame) {
              a.px[ga] = pa[0]; a.py[ga] = pa[1]; a.pz[ga] = pa[2];
              a.px[gb] = pb[0]; a.py[gb] = pb[1]; a.pz[gb] = pb[2];
            } else {  // the stored value plus the increment
              a.px[ga] += (S)(pa[0] - pa0[0]); a.py[ga] += (S)(pa[1] - pa0[1]); a.pz[ga] += (S)(pa[2] - pa0[2]);
              a.px[gb] += (S)(pb[0] - pb0[0]); a.py[gb] += (S)(pb[1] - pb0[1]); a.pz[gb] += (S)(pb[2] - pb0[2]);
            }
            bad |= !isfinite(a.eps[ga]) || !isfinite(a.eps[gb]);
          }
          ++n_tot;
          n_acc += dcs == 0;
          n_rb += dcs == 1;
          n_rm += dcs == 2;
          if (recs) {
            const unsigned long long sr = atomicAdd(rec_count, 1ull);
            if ((int64_t)sr < rec_cap) {
              sdpd_pair_rec rc;
              rc.id_i = a.id[ga];
              rc.id_j = a.id[gb];
              rc.colour = colour;
              rc.owner = (int32_t)o;
              rc.decision = dcs;
              rc.level = seq;  // position in the sequential order
              rc.margin = margin;
              rc.margin_lo = A::mixed ? (double)m32 : margin;
              rc.margin_tol = (double)tol;
              recs[sr] = rc;
            }
          }
        }
        ++seq;
        __syncwarp();
      }
    }
  }
  // pressure over rho^2 of the new energies, Eq. (pg-eos)
  const S pi_coef = (S)(c.c_rho / (c.C_K * c.m));
  for (int q = lane; q < nb; q += 32) {
    const int g = perm[q];
    qp4[g].w = (S)a.eps[g] * pi_coef / a.rho[g];
  }
  __syncwarp();
  return BigCounts{n_tot, n_acc, n_rb, n_rm, (int)negative, (int)bad};
}

// Block schedule of a colour launch: OPW blocks per warp (each on 32 / OPW
// lanes) and W warps per thread block.  Every variant runs the same pair
// updates in the same per-particle order, so the results are identical; only
// the mapping onto the GPU differs.  Register budget: 128 per thread for the
// mixed path (16 warps per SM), none for float64.
template <class P, int W>
constexpr int fd_min_blocks() { return P::mixed ? 16 / W : (W >= 4 ? 1 : 4 / W); }

// P is the storage policy of the state arrays, A the arithmetic policy of
// the pair updates: A = P except for a float64 state swept with float32
// pair arithmetic (P = Fp64, A = Mixed), where momenta and energies go back
// as their float64 values plus the float32 increments of the visit.
template <class P, class A, int KIND, int OPW, int W>
__global__ void __launch_bounds__(W * 32, fd_min_blocks<A, W>())
    k_fd_colour(Consts c, FDConst<typename A::R> k, Arrays<P> a, typename P::V4* __restrict__ qp4,
                const typename P::V4* __restrict__ qr4,
                const int32_t* __restrict__ cell_start, const int32_t* __restrict__ mrank,
                const uint32_t* __restrict__ xmx, const uint32_t* __restrict__ xmy,
                const uint32_t* __restrict__ xmz, const uint32_t* __restrict__ hdr,
                const uint16_t* __restrict__ lvl, const uint16_t* __restrict__ pairs, int colour, uint64_t seed,
                const unsigned long long* __restrict__ sweep_ptr, unsigned long long* counters, int* status,
                sdpd_pair_rec* recs, unsigned long long* rec_count, int64_t rec_cap, unsigned* __restrict__ queue,
                const int32_t* __restrict__ order, int32_t* __restrict__ big_perm,
                const int2* __restrict__ big_list, const uint32_t* __restrict__ big_count) {
  using R = typename A::R;  // pair arithmetic
  using S = typename P::R;  // stored momenta, densities, geometry
  constexpr bool kSame = std::is_same<R, S>::value;
  constexpr int kGroupLanes = 32 / OPW;
  __shared__ FdSmem<R> sm_all[W][OPW];
  const uint64_t sweep = *sweep_ptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / kGroupLanes, gl = lane % kGroupLanes;
  const int hx = c.nc[0] >> 1, hy = c.nc[1] >> 1, hz = c.nc[2] >> 1;
  const int64_t nown = (int64_t)hx * hy * hz;
  FdSmem<R>& sm = sm_all[warp][grp];
  const S inv_h = (S)(1.0 / c.h), cF = (S)c.cF;
  const S pi_coef = (S)(c.c_rho / (c.C_K * c.m));
  unsigned n_tot = 0, n_rb = 0, n_rm = 0;  // per lane (accepted = total - rejected)
  bool negative = false, bad = false;
  // The grid holds as many thread blocks as fit on the GPU at once; each
  // warp takes the colour's blocks OPW at a time from queue[0] until they
  // run out, so no partial last wave of thread blocks idles the GPU and
  // blocks of uneven depth balance out.  The blocks come in the order of
  // `order` (deepest first), so the blocks a warp runs in lockstep have
  // similar depth.  queue[1] counts the warps that are done; the last one
  // sets them back to zero for the next launch (queue[2]: the next entry of
  // the colour's list of blocks beyond capacity).
  for (;;) {
    unsigned w0 = 0;
    if (lane == 0) w0 = atomicAdd(queue, (unsigned)OPW);
    w0 = __shfl_sync(0xffffffffu, w0, 0);
    if ((int64_t)w0 >= nown) break;
    const int64_t wi = (int64_t)w0 + grp;
    const int64_t w = wi < nown ? (int64_t)order[colour * nown + wi] : nown;
    int np = 0, nlev = 0;
    int64_t o = 0;
    int ox = 0, oy = 0, oz = 0;
    if (w < nown) {
      ox = 2 * (int)(w % hx) + (colour & 1);
      oy = 2 * (int)((w / hx) % hy) + ((colour >> 1) & 1);
      oz = 2 * (int)(w / ((int64_t)hx * hy)) + ((colour >> 2) & 1);
      o = ox + (int64_t)c.nc[0] * (oy + (int64_t)c.nc[1] * oz);
      const uint32_t hd = hdr[o];
      if (hd != kHdrBig) {  // (a block beyond capacity was swept above)
        np = (int)(hd & 0xffffu);
        nlev = (int)(hd >> 16);
      }
    }
    BlockCells b;
    b.base[8] = 0;
    if (np > 0) block_cells(c, ox, oy, oz, mrank, cell_start, b);
    const int nb = np > 0 ? b.base[8] : 0;
    BlockGeom<P> geo;
    geo.init(c, ox, oy, oz, xmx, xmy, xmz);
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (gl == t) {
        sm.cst[t] = b.start[t];
        sm.cbs[t] = b.base[t];
      }
    __syncwarp();
    // storage index of block particle q (recomputed where needed, which keeps
    // shared memory small enough for eight thread blocks per SM)
    auto gidx = [&](int q) {
      int d = 0;
#pragma unroll
      for (int t = 1; t < 8; ++t) d += (q >= sm.cbs[t]);
      return sm.cst[d] + (q - sm.cbs[d]);
    };
    // the same, also giving the particle's cell in the block
    auto gidx_code = [&](int q, int& d) {
      d = 0;
#pragma unroll
      for (int t = 1; t < 8; ++t) d += (q >= sm.cbs[t]);
      return sm.cst[d] + (q - sm.cbs[d]);
    };
    for (int q = gl; q < nb; q += kGroupLanes) {
      const int g = gidx(q);
      sm.px[q] = a.px[g]; sm.py[q] = a.py[g]; sm.pz[q] = a.pz[g];
      if constexpr (A::mixed) {
        sm.es[q] = (float)a.eps[g];
        sm.ec[q] = 0.0f;
      } else {
        sm.e[q] = a.eps[g];
      }
    }
    for (int L = gl; L <= nlev; L += kGroupLanes) sm.off[L] = lvl[o * (kMaxLevels + 1) + L];
    __syncwarp();
    const uint16_t* off = sm.off;
    const uint16_t* pl = pairs + o * kMaxPairs;
    int L = 0, pos = 0;
    while (__any_sync(0xffffffffu, pos < np)) {
      // stage pairs [cbeg, cend) of the level-ordered list; the chunk ends on
      // a level boundary when at least one whole level fits, so that no level
      // is split over two chunks (a split level costs an extra round)
      const int cbeg = pos;
      int cend = min(pos + kChunk, np);
      if (pos < np && (int)off[L + 1] <= cend) {
        int Le = L + 1;
        while (Le < nlev && (int)off[Le + 1] <= cend) ++Le;
        cend = off[Le];
      }
      for (int t = cbeg + gl; t < cend; t += kGroupLanes) {
        const uint16_t pr = pl[t];
        const int ia = pr & 255, ib = pr >> 8;  // ia holds the lower id
        int da, db;
        const int ga = gidx_code(ia, da), gb = gidx_code(ib, db);
        S xa, ya, za, xb, yb, zb, rx, ry, rz;
        // positions and densities of the latest density pass (one load each)
        const typename P::V4 qa = ld4(&qr4[ga]), qb = ld4(&qr4[gb]);
        geo.local(qa, da, xa, ya, za);
        geo.local(qb, db, xb, yb, zb);
        geo.disp(xa, ya, za, xb, yb, zb, rx, ry, rz);
        const S r2 = r2_of(rx, ry, rz);
        const S inv_r = fm::rsqrt(r2);
        const int slot = t - cbeg;
        sm.pr[slot] = pr;
        sm.ex[slot] = (R)(rx * inv_r);
        sm.ey[slot] = (R)(ry * inv_r);
        sm.ez[slot] = (R)(rz * inv_r);
        sm.base[slot] = (R)fm::div(kernel_F<KIND>(r2 * inv_r * inv_h, cF), qa.w * qb.w);
        R G[3], U;
        pair_randoms_fast(seed, sweep, (uint64_t)a.id[ga], (uint64_t)a.id[gb], G, &U);
        sm.G0[slot] = G[0]; sm.G1[slot] = G[1]; sm.G2[slot] = G[2];
        sm.lnU[slot] = k.scheme == SDPD_SCHEME_EMS ? fm::log(U) : U;  // off the pairs' dependency chain
      }
      __syncwarp();
      // the chunk's levels, or parts of them
      bool more = cbeg < cend;
      while (__any_sync(0xffffffffu, more)) {
        int lb = 0, le = 0;
        if (more) {
          lb = max((int)off[L], cbeg);
          le = min((int)off[L + 1], cend);
        }
        for (int t = lb + gl; t < le; t += kGroupLanes) {
          const int slot = t - cbeg;
          const uint16_t pr = sm.pr[slot];
          const int ia = pr & 255, ib = pr >> 8;
          R pa[3] = {sm.px[ia], sm.py[ia], sm.pz[ia]};
          R pb[3] = {sm.px[ib], sm.py[ib], sm.pz[ib]};
          const R G[3] = {sm.G0[slot], sm.G1[slot], sm.G2[slot]};
          double margin;
          float m32 = 0.0f, tol = 0.0f;
          int dcs;
          if constexpr (A::mixed) {
            const float eaf = sm.es[ia], ebf = sm.es[ib];
            // rare (near ties of the bound or the ratio): the two energies in
            // float64, and the pair's uniform drawn again
            auto exact_e = [&](double& ea, double& eb) {
              const double ga = a.eps[gidx(ia)], gb = a.eps[gidx(ib)];
              ea = ga + (((double)eaf - (double)(float)ga) + (double)sm.ec[ia]);
              eb = gb + (((double)ebf - (double)(float)gb) + (double)sm.ec[ib]);
            };
            auto uniform = [&]() {
              R Gr[3], U;
              pair_randoms_fast(seed, sweep, (uint64_t)a.id[gidx(ia)], (uint64_t)a.id[gidx(ib)], Gr, &U);
              return U;
            };
            float dh, dl;
            dcs = fd_pair_mixed(k, sm.ex[slot], sm.ey[slot], sm.ez[slot], sm.base[slot], G, uniform,
                                sm.lnU[slot], pa, pb, eaf, ebf, exact_e, dh, dl, margin, m32, tol,
                                recs != nullptr, negative);
            if (dcs == 0) {
              sm.px[ia] = pa[0]; sm.py[ia] = pa[1]; sm.pz[ia] = pa[2];
              sm.px[ib] = pb[0]; sm.py[ib] = pb[1]; sm.pz[ib] = pb[2];
              float s, e;
              eft::two_sum(eaf, dh, s, e);
              sm.ec[ia] = __fadd_rn(sm.ec[ia], __fadd_rn(e, dl));
              sm.es[ia] = s;
              eft::two_sum(ebf, dh, s, e);
              sm.ec[ib] = __fadd_rn(sm.ec[ib], __fadd_rn(e, dl));
              sm.es[ib] = s;
              bad |= !isfinite(sm.es[ia]) || !isfinite(sm.es[ib]);
            }
          } else {
            const double ea = sm.e[ia], eb = sm.e[ib];
            double deps;
            dcs = fd_pair(k, sm.ex[slot], sm.ey[slot], sm.ez[slot], sm.base[slot], G, sm.lnU[slot], pa, pb, ea,
                          eb, deps, margin, negative);
            if (dcs == 0) {
              sm.px[ia] = pa[0]; sm.py[ia] = pa[1]; sm.pz[ia] = pa[2];
              sm.px[ib] = pb[0]; sm.py[ib] = pb[1]; sm.pz[ib] = pb[2];
              sm.e[ia] = ea + deps;
              sm.e[ib] = eb + deps;
              bad |= !isfinite(sm.e[ia]) || !isfinite(sm.e[ib]);
            }
          }
          ++n_tot;
          n_rb += dcs == 1;
          n_rm += dcs == 2;
          if (recs) {
            const unsigned long long s = atomicAdd(rec_count, 1ull);
            if ((int64_t)s < rec_cap) {
              sdpd_pair_rec rc;
              rc.id_i = a.id[gidx(ia)];
              rc.id_j = a.id[gidx(ib)];
              rc.colour = colour;
              rc.owner = (int32_t)o;
              rc.decision = dcs;
              rc.level = L;
              rc.margin = margin;
              rc.margin_lo = A::mixed ? (double)m32 : margin;
              rc.margin_tol = (double)tol;
              recs[s] = rc;
            }
          }
        }
        __syncwarp();
        if (more) {
          if ((int)off[L + 1] <= cend) {  // level L done
            ++L;
            more = L < nlev && (int)off[L] < cend;
          } else {
            more = false;  // level L continues in the next chunk
          }
        }
      }
      pos = cend;
      __syncwarp();
    }
    for (int q = gl; q < nb; q += kGroupLanes) {
      const int g = gidx(q);
      if constexpr (kSame) {
        a.px[g] = sm.px[q]; a.py[g] = sm.py[q]; a.pz[g] = sm.pz[q];
      } else {  // the stored value plus this visit's increment
        a.px[g] += (S)(sm.px[q] - (R)a.px[g]);
        a.py[g] += (S)(sm.py[q] - (R)a.py[g]);
        a.pz[g] += (S)(sm.pz[q] - (R)a.pz[g]);
      }
      double e;
      if constexpr (A::mixed) {  // once per visit: the load value plus the visit's exact change
        const double e0 = a.eps[g];
        e = e0 + (((double)sm.es[q] - (double)(float)e0) + (double)sm.ec[q]);
      }
      else e = sm.e[q];
      a.eps[g] = e;
      // pressure over rho^2 of the new energy, Eq. (pg-eos): pi = c_rho eps / (C_K m rho)
      // (from the stored float64 energy, as a restart recomputes it)
      qp4[g].w = (S)e * pi_coef / a.rho[g];
    }
    __syncwarp();  // the group's shared memory is refilled by the next block
  }
  // the colour's blocks beyond capacity (listed by the schedule), swept pair
  // by pair by whole warps once the queue is empty
  for (;;) {
    unsigned bi = 0;
    if (lane == 0) bi = atomicAdd(&queue[2], 1u);
    bi = __shfl_sync(0xffffffffu, bi, 0);
    if (bi >= big_count[colour]) break;
    const int2 ent = big_list[colour * nown + bi];
    const int64_t ob = ent.x;
    int bx, by, bz;
    owner_coords(c, ob, bx, by, bz);
    const BigCounts bc = fd_big_block<P, A, KIND>(c, k, a, qp4, cell_start, mrank, xmx, xmy, xmz, ob, bx, by, bz,
                                                  colour, seed, sweep, recs, rec_count, rec_cap, big_perm + ent.y);
    unsigned long long bt = bc.tot, ba = bc.acc, bb = bc.rb, bm = bc.rm;  // (rare: counted at once)
    for (int s = 16; s > 0; s >>= 1) {
      bt += __shfl_xor_sync(0xffffffffu, bt, s);
      ba += __shfl_xor_sync(0xffffffffu, ba, s);
      bb += __shfl_xor_sync(0xffffffffu, bb, s);
      bm += __shfl_xor_sync(0xffffffffu, bm, s);
    }
    if (lane == 0 && bt) {
      atomicAdd(&counters[0], bt);
      atomicAdd(&counters[1], ba);
      atomicAdd(&counters[2], bb);
      atomicAdd(&counters[3], bm);
    }
    negative |= bc.negative != 0;
    bad |= bc.bad != 0;
  }
  if (lane == 0) {
    const unsigned total = gridDim.x * (unsigned)W;
    __threadfence();  // this warp's last take from queue[0] is performed before it counts as done
    if (atomicAdd(&queue[1], 1u) == total - 1u) {  // every warp has taken its last block
      queue[0] = 0u;
      queue[1] = 0u;
      queue[2] = 0u;
    }
  }
  // counters
  unsigned long long c_tot = n_tot, c_rb = n_rb, c_rm = n_rm, c_acc = n_tot - n_rb - n_rm;
  for (int s = 16; s > 0; s >>= 1) {
    c_tot += __shfl_xor_sync(0xffffffffu, c_tot, s);
    c_acc += __shfl_xor_sync(0xffffffffu, c_acc, s);
    c_rb += __shfl_xor_sync(0xffffffffu, c_rb, s);
    c_rm += __shfl_xor_sync(0xffffffffu, c_rm, s);
  }
  const unsigned any_neg = __any_sync(0xffffffffu, negative), any_bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    if (c_tot) {
      atomicAdd(&counters[0], c_tot);
      atomicAdd(&counters[1], c_acc);
      atomicAdd(&counters[2], c_rb);
      atomicAdd(&counters[3], c_rm);
    }
    if (any_neg) atomicOr(status, kStNegative);
    if (any_bad) atomicOr(status, kStNaN);
  }
}

template <class R>
static FDConst<R> fd_const(const Consts& c, double dt) {
  FDConst<R> k;
  k.m = (R)c.m;
  k.inv_m = (R)(1.0 / c.m);
  k.half_m = (R)(0.5 * c.m);
  k.inv_h = (R)(1.0 / c.h);
  k.cF = (R)c.cF;
  k.kpar_m2 = (R)c.kpar_m2;
  k.kperp_m2 = (R)c.kperp_m2;
  k.inv_C_K = (R)(1.0 / c.C_K);
  k.kB = (R)c.kB;
  k.two_over_CK = (R)(2.0 / c.C_K);
  k.dt_over_m = (R)(dt / c.m);
  k.CKm1 = (R)(c.C_K / c.kB - 1.0);
  k.four_kB_over_m = (R)(4.0 * c.kB / c.m);
  k.CKm1_d = c.C_K / c.kB - 1.0;
  k.nq_hi = (float)(-0.25 / c.m);
  k.nq_lo = (float)(-0.25 / c.m - (double)k.nq_hi);
  k.scheme = c.scheme;
  return k;
}

// Thread blocks of a colour kernel that the device holds at once (SMs x
// blocks per SM, from the occupancy calculator; at least one), computed once
// per kernel on the device current at the first launch.
template <class P, class A, int KIND, int OPW, int W>
int fd_resident_blocks() {
  static const int n = [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fd_colour<P, A, KIND, OPW, W>, W * 32, 0);
    return std::max(1, sms) * std::max(1, per_sm);
  }();
  return n;
}

// A block schedule fits when its groups' shared memory stays within the 48 KB
// a thread block may declare statically.
template <class P, int OPW, int W>
constexpr bool fd_fits() { return sizeof(FdSmem<typename P::R>) * OPW * W <= 48 * 1024; }

constexpr int kFdOpw[kFdVariants] = {2, 2, 1, 1, 1};
constexpr int kFdWarps[kFdVariants] = {2, 1, 1, 2, 4};

// One colour launch with block-schedule variant (OPW, W); a schedule that
// does not fit runs as variant 1.
template <class P, class A, int KIND, int OPW, int W>
void launch_colour(const Consts& c, const FDConst<typename A::R>& k, const Arrays<P>& a, const Workspace& w,
                   int col, uint64_t seed, sdpd_pair_rec* recs, cudaStream_t s) {
  if constexpr (!fd_fits<A, OPW, W>()) {
    launch_colour<P, A, KIND, 2, 1>(c, k, a, w, col, seed, recs, s);
  } else {
    const int64_t nown = (int64_t)(c.nc[0] / 2) * (c.nc[1] / 2) * (c.nc[2] / 2);
    const int64_t per_block = (int64_t)W * OPW;
    const int64_t need = (nown + per_block - 1) / per_block;
    const int64_t resident = (int64_t)fd_resident_blocks<P, A, KIND, OPW, W>();
    const unsigned gf = (unsigned)std::max<int64_t>(1, std::min(need, resident));
    k_fd_colour<P, A, KIND, OPW, W><<<gf, W * 32, 0, s>>>(
        c, k, a, (typename P::V4*)w.qp4, (const typename P::V4*)w.qr4, w.cell_start, w.mrank, w.xmin[0], w.xmin[1], w.xmin[2], w.sched_hdr,
        w.sched_lvl, w.sched_pair, col, seed, w.sweep, w.counters, w.status, recs, w.pair_rec_count,
        w.pair_rec_cap, w.fd_queue + 3 * col, w.blk_order, w.big_perm, w.big_list, w.big_count);
  }
}

// The eight colour launches of one sweep.  variant indexes the block
// schedules (blocks per warp, warps per thread block):
// 0 (2, 2), 1 (2, 1), 2 (1, 1), 3 (1, 2), 4 (1, 4).
template <class P, class A, int KIND>
void launch_colours_kind(const Consts& c, const Workspace& w, int cur, double dt, uint64_t seed, int record,
                         int variant, cudaStream_t s) {
  const FDConst<typename A::R> k = fd_const<typename A::R>(c, dt);
  const Arrays<P> a = view<P>(w, cur);
  sdpd_pair_rec* recs = record ? w.pair_recs : nullptr;
  for (int col = 0; col < 8; ++col) {
    switch (variant) {
      case 0: launch_colour<P, A, KIND, 2, 2>(c, k, a, w, col, seed, recs, s); break;
      case 1: launch_colour<P, A, KIND, 2, 1>(c, k, a, w, col, seed, recs, s); break;
      case 2: launch_colour<P, A, KIND, 1, 1>(c, k, a, w, col, seed, recs, s); break;
      case 3: launch_colour<P, A, KIND, 1, 2>(c, k, a, w, col, seed, recs, s); break;
      default: launch_colour<P, A, KIND, 1, 4>(c, k, a, w, col, seed, recs, s); break;
    }
  }
}

// Fills the resident-block counts of every block schedule ahead of time (a
// host query, kept out of stream captures).
template <class P, class A>
void fd_prepare() {
  fd_resident_blocks<P, A, SDPD_KERNEL_LUCY, 2, 2>();
  fd_resident_blocks<P, A, SDPD_KERNEL_LUCY, 2, 1>();
  fd_resident_blocks<P, A, SDPD_KERNEL_LUCY, 1, 1>();
  fd_resident_blocks<P, A, SDPD_KERNEL_LUCY, 1, 2>();
  fd_resident_blocks<P, A, SDPD_KERNEL_LUCY, 1, 4>();
  fd_resident_blocks<P, A, SDPD_KERNEL_CUBIC, 2, 2>();
  fd_resident_blocks<P, A, SDPD_KERNEL_CUBIC, 2, 1>();
  fd_resident_blocks<P, A, SDPD_KERNEL_CUBIC, 1, 1>();
  fd_resident_blocks<P, A, SDPD_KERNEL_CUBIC, 1, 2>();
  fd_resident_blocks<P, A, SDPD_KERNEL_CUBIC, 1, 4>();
}

template <class P, class A>
void launch_fd_colours(const Consts& c, const Workspace& w, int cur, double dt, uint64_t seed, int record,
                       cudaStream_t s) {
  if (c.N == 0) return;
  int variant = c.fd_variant;
  if (variant < 0 || variant >= kFdVariants) variant = fd_default_variant(A::mixed);
  if (c.kernel == SDPD_KERNEL_LUCY)
    launch_colours_kind<P, A, SDPD_KERNEL_LUCY>(c, w, cur, dt, seed, record, variant, s);
  else
    launch_colours_kind<P, A, SDPD_KERNEL_CUBIC>(c, w, cur, dt, seed, record, variant, s);
}

}  // namespace sdpd
