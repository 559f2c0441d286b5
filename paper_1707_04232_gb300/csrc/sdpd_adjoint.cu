// sdpd_adjoint.cu -- reverse-mode passes of the conservative dynamics
// (float64 storage layout only): the pull-back of a kick through the forces
// of Eq. (cons-forces), the pressures of Eq. (pg-eos) at fixed entropy
// (Section 3.1) and the density sum of Eq. (sdpd-rho-v) with its gradient,
// Eq. (gradient-rho); and the gradient of the virial pressure.
//
// A pair sum Phi = wt sum_{i<j} m^2 (pi_i + pi_j) F(r_ij) t_ij, with
// t_ij = (v_i - v_j) . r_ij (a kick pulled back along v) or |r_ij|^2 (the
// virial), is differentiated in two neighbour-list passes around one
// elementwise step:
//   pass A  A_i = m^2 sum_j F(r_ij) t_ij             (dPhi/dpi_i = wt A_i)
//   mid     rbar_i = dL/drho_i through pi_i (and the energy terms), the
//           entropy / energy and parameter cotangents
//   pass B  dL/dq_i = sum_j [ c_ij (F'/r t_ij r_ij + F dt_ij/dq_i)
//                             - m F (rbar_i + rbar_j) r_ij ],  c_ij = wt m^2 (pi_i + pi_j)
//           and dL/dh = sum_{i<j} [ c_ij t_ij dF/dh + m dW/dh (rbar_i + rbar_j) ]
//                       + sum_i rbar_i m dW/dh(0).
// Each pass is a gather over the neighbour list of particle i (one thread per
// particle, no atomics); every pair is met from both sides, so the symmetric
// h terms are halved.  Cotangents of particles are kept in id order.
#include <math.h>

#include "sdpd_internal.cuh"

namespace sdpd {

namespace {

// dF/dr: Lucy -2 cF (1 - x)/h; cubic -3 cF/h (x <= 1/2), -(cF/h)(1 - x)(1 + x)/x^2
template <int KIND>
__device__ __forceinline__ double kernel_dF(double x, double cF, double inv_h) {
  if (KIND == SDPD_KERNEL_LUCY) return -2.0 * cF * (1.0 - x) * inv_h;
  if (x <= 0.5) return -3.0 * cF * inv_h;
  return -cF * inv_h * (1.0 - x) * (1.0 + x) / (x * x);
}

// Displacement r_ij with the periodic image taken from the neighbour-list
// entry's stencil code (offset + 1 per axis, 2 bits each) and the home cell.
struct Images {
  double m[3], p[3];  // shifts of the offsets -1 and +1 per axis
  __device__ void init(const Consts& c, double cellbits_w) {
    int ci[3];
    unpack_cell(w_to_cellbits(cellbits_w), ci[0], ci[1], ci[2]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      m[d] = image_shift(ci[d], -1, c.nc[d], c.L[d]);
      p[d] = image_shift(ci[d], 1, c.nc[d], c.L[d]);
    }
  }
};

__device__ __forceinline__ void pair_disp(const Images& im, uint32_t code, const D4& qi, const D4& qj, double& dx,
                                          double& dy, double& dz) {
  double d[3] = {__dsub_rn(qi.x, qj.x), __dsub_rn(qi.y, qj.y), __dsub_rn(qi.z, qj.z)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const uint32_t k = (code >> (2 * a)) & 3u;
    const double s = k == 0 ? im.m[a] : (k == 2 ? im.p[a] : 0.0);
    if (s != 0.0) d[a] = __dadd_rn(d[a], s);
  }
  dx = d[0]; dy = d[1]; dz = d[2];
}

// v_i = scale * pbar[id_i], rbar slot cleared
__global__ void k_adj_gather(int64_t N, const int32_t* __restrict__ id, const double* __restrict__ pbar,
                             double scale, D4* __restrict__ vs4) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t k = id[i];
  st4(&vs4[i], D4{scale * pbar[3 * k], scale * pbar[3 * k + 1], scale * pbar[3 * k + 2], 0.0});
}

// pass A: A_i = m^2 sum_j F(r_ij) t_ij
template <int KIND, int MODE>
__global__ void __launch_bounds__(128) k_adj_pairsum(Consts c, const D4* __restrict__ qp4, const D4* __restrict__ q4,
                                                     const D4* __restrict__ vs4, const uint32_t* __restrict__ nlist,
                                                     const int32_t* __restrict__ nn, double* __restrict__ A,
                                                     int* __restrict__ status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= c.N) return;
  const D4 qi = ld4(&qp4[i]);
  Images im;
  im.init(c, q4[i].w);
  D4 vi{0.0, 0.0, 0.0, 0.0};
  if (MODE == 0) vi = ld4(&vs4[i]);
  const double inv_h = 1.0 / c.h;
  double acc = 0.0;
  int n = nn[i];
  if (n > c.nbr_cap) {  // the gradient passes walk the list only
    atomicOr(status, kStNbrCap);
    n = c.nbr_cap;
  }
#pragma unroll 2
  for (int k = 0; k < n; ++k) {
    const uint32_t e = __ldg(&nlist[nbr_slot(i, k, c.nbr_cap)]);
    const D4 qj = ld4(&qp4[e >> 6]);
    double dx, dy, dz;
    pair_disp(im, e & 63u, qi, qj, dx, dy, dz);
    const double r2 = r2_of(dx, dy, dz);
    double t;
    if (MODE == 0) {
      const D4 vj = ld4(&vs4[e >> 6]);
      t = (vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz;
    } else {
      t = r2;
    }
    acc += kernel_F<KIND>(pair_r(r2) * inv_h, c.cF) * t;
  }
  A[i] = c.m * c.m * acc;
}

// Elementwise step of the trajectory's reverse pass at position k (state
// after the sweep increments of step k - 1).  Pressures pi = c_rho eps /
// (C_K m rho); at fixed entropy (eps = E(S, rho))
//   dpi/drho = pi (c_rho/C_K - 1)/rho, dpi/dS = pi/C_K,
//   dpi/dc_rho = pi (1/c_rho + ln rho / C_K), dpi/dC_K = -pi (1 + ln eps)/C_K.
// KICK1 (k < n): first kick of step k at S_k, with eps_k; then the entropy
//   S_k = C_K ln eps_k - c_rho ln rho_k carries Sbar_cur (complete now) to
//   eps_k and rho_k.  Without KICK1 the cotangent of eps_k is epsbar_n.
// KICK2 (k > 0): second kick of step k - 1 at S_{k-1}, with the energies
//   before the increments, eps'_k = eps_k - deps_{k-1}, and the final
//   energies eps'_k = E(S_{k-1}, rho_k) (the increments pass cotangents
//   through); they start Sbar_prev, the entropy cotangent of step k - 1.
// Both kicks pull back along the same v, so the pair pass that follows uses
// the summed pressures (written to qp4.w) and rbar (vs4.w).
constexpr int kAdjKick1 = 1;
constexpr int kAdjKick2 = 2;

__global__ void k_adj_mid_step(Consts c, D4* __restrict__ qp4, const double* __restrict__ rho,
                               const double* __restrict__ eps, const int32_t* __restrict__ id,
                               const double* __restrict__ A, int flags, const double* __restrict__ deps_prev,
                               double* __restrict__ Sbar_cur, double* __restrict__ Sbar_prev,
                               const double* __restrict__ epsbar_n, double* __restrict__ epsbar0,
                               D4* __restrict__ vs4, double* __restrict__ thbar) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= c.N) return;
  const int64_t k = id[i];
  const double CK = c.C_K, cr = c.c_rho, r = rho[i], lr = log(r);
  const double pif = cr / (CK * c.m * r);  // pi per unit energy
  const double a_i = A ? A[i] : 0.0;
  double rb = 0.0, tcr = 0.0, tck = 0.0, pisum = 0.0, ge;
  if (flags & kAdjKick1) {
    const double e = eps[i], le = log(e), pi = e * pif, g = a_i * pi;
    const double sb = Sbar_cur[k] + g / CK;
    rb += g * (cr / CK - 1.0) / r;
    tcr += g * (1.0 / cr + lr / CK);
    tck -= g * (1.0 + le) / CK;
    pisum += pi;
    ge = sb * CK / e;  // S_k = C_K ln eps_k - c_rho ln rho_k
    rb -= sb * cr / r;
    tcr -= sb * lr;
    tck += sb * le;
  } else {
    ge = epsbar_n ? epsbar_n[k] : 0.0;
  }
  if (flags & kAdjKick2) {
    const double e = eps[i] - deps_prev[k], le = log(e), pi = e * pif, g = a_i * pi;
    const double gf = ge * e / CK;  // eps' = E(S_{k-1}, rho_k)
    rb += gf * cr / r + g * (cr / CK - 1.0) / r;
    tcr += gf * lr + g * (1.0 / cr + lr / CK);
    tck -= gf * le + g * (1.0 + le) / CK;
    pisum += pi;
    Sbar_prev[k] = gf + g / CK;
  }
  if (epsbar0) epsbar0[k] = ge;
  thbar[3 * k + 1] += tcr;
  thbar[3 * k + 2] += tck;
  vs4[i].w = rb;
  qp4[i].w = pisum;
}

// Recording a step with its sweep frozen: the increments d = after - before
// of the momenta and energies (id order) are stored, and the state is set to
// before + d, the value a replay that adds d reproduces bit for bit.  The
// pressure the next first kick uses, pi = c_rho eps / (C_K m rho) (Eq.
// pg-eos), is recomputed from the stored energy, as the replay does.
__global__ void k_adj_freeze(int64_t N, double pi_coef, const int32_t* __restrict__ id, double* __restrict__ px,
                             double* __restrict__ py, double* __restrict__ pz, double* __restrict__ eps,
                             const double* __restrict__ rho, D4* __restrict__ qp4, const double* __restrict__ pre,
                             double* __restrict__ dp, double* __restrict__ de) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t k = id[i];
  double* v[4] = {px, py, pz, eps};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const double b = pre[a * N + i], d = v[a][i] - b;
    v[a][i] = b + d;
    if (a < 3) dp[3 * k + a] = d;
    else de[k] = d;
  }
  qp4[i].w = eps[i] * pi_coef / rho[i];
}

// Replaying a frozen step: the stored increments added to the state, and
// the pressures recomputed from the new energies.
__global__ void k_adj_increment(int64_t N, double pi_coef, const int32_t* __restrict__ id, double* __restrict__ px,
                                double* __restrict__ py, double* __restrict__ pz, double* __restrict__ eps,
                                const double* __restrict__ rho, D4* __restrict__ qp4, const double* __restrict__ dp,
                                const double* __restrict__ de) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t k = id[i];
  px[i] = px[i] + dp[3 * k];
  py[i] = py[i] + dp[3 * k + 1];
  pz[i] = pz[i] + dp[3 * k + 2];
  const double e = eps[i] + de[k];
  eps[i] = e;
  qp4[i].w = e * pi_coef / rho[i];
}

// Elementwise step of the virial pressure's gradient at fixed energies:
// dpi/drho = -pi/rho, dpi/deps = pi/eps, dpi/dc_rho = pi/c_rho,
// dpi/dC_K = -pi/C_K.  val_id receives wt (|p|^2/m + pi A), whose sum is the
// virial pressure.
__global__ void k_adj_mid_virial(Consts c, const D4* __restrict__ qp4, const double* __restrict__ rho,
                                 const double* __restrict__ eps, const double* __restrict__ px,
                                 const double* __restrict__ py, const double* __restrict__ pz,
                                 const int32_t* __restrict__ id, const double* __restrict__ A, double wt,
                                 D4* __restrict__ vs4, double* __restrict__ val_id, double* __restrict__ gp,
                                 double* __restrict__ geps, double* __restrict__ thbar) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= c.N) return;
  const int64_t k = id[i];
  const double pi = qp4[i].w, a = A[i];
  const double x = px[i], y = py[i], z = pz[i];
  val_id[k] = wt * ((x * x + y * y + z * z) / c.m + pi * a);
  const double g = wt * a * pi;
  if (gp) {
    const double s = 2.0 * wt / c.m;
    gp[3 * k] = s * x;
    gp[3 * k + 1] = s * y;
    gp[3 * k + 2] = s * z;
    geps[k] = g / eps[i];
    thbar[3 * k] = 0.0;
    thbar[3 * k + 1] = g / c.c_rho;
    thbar[3 * k + 2] = -g / c.C_K;
  }
  vs4[i].w = -g / rho[i];
}

// pass B (MODE 0: kick pulled back along v; 1: virial; 2: density term only)
template <int KIND, int MODE>
__global__ void __launch_bounds__(128) k_adj_back(Consts c, const D4* __restrict__ qp4, const D4* __restrict__ q4,
                                                  const D4* __restrict__ vs4, const int32_t* __restrict__ id,
                                                  const uint32_t* __restrict__ nlist,
                                                  const int32_t* __restrict__ nn, double wt, int accumulate,
                                                  double* __restrict__ qbar, double* __restrict__ thbar,
                                                  int* __restrict__ status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= c.N) return;
  const D4 qi = ld4(&qp4[i]);
  const D4 vi = ld4(&vs4[i]);
  Images im;
  im.init(c, q4[i].w);
  const double inv_h = 1.0 / c.h, m = c.m, cm2 = wt * c.m * c.m;
  double gx = 0.0, gy = 0.0, gz = 0.0, gh = 0.0;
  int n = nn[i];
  if (n > c.nbr_cap) {  // the gradient passes walk the list only
    atomicOr(status, kStNbrCap);
    n = c.nbr_cap;
  }
#pragma unroll 2
  for (int k = 0; k < n; ++k) {
    const uint32_t e = __ldg(&nlist[nbr_slot(i, k, c.nbr_cap)]);
    const D4 qj = ld4(&qp4[e >> 6]);
    const D4 vj = ld4(&vs4[e >> 6]);
    double dx, dy, dz;
    pair_disp(im, e & 63u, qi, qj, dx, dy, dz);
    const double r2 = r2_of(dx, dy, dz);
    const double r = pair_r(r2), x = r * inv_h;
    const double f = kernel_F<KIND>(x, c.cF);
    const double rb = vi.w + vj.w;
    // density: d rho / d q along r_ij, and dW/dh = (r^2 F - 3 W)/h
    double s = -m * f * rb;
    gh += m * (r2 * f - 3.0 * kernel_W<KIND>(x, c.cW)) * inv_h * rb;
    if (MODE != 2) {
      const double fp = kernel_dF<KIND>(x, c.cF, inv_h);
      const double cc = cm2 * (qi.w + qj.w);
      double t, ux, uy, uz;
      if (MODE == 0) {
        ux = vi.x - vj.x; uy = vi.y - vj.y; uz = vi.z - vj.z;
        t = ux * dx + uy * dy + uz * dz;
      } else {
        ux = 2.0 * dx; uy = 2.0 * dy; uz = 2.0 * dz;
        t = r2;
      }
      // F'/r t vanishes with r at coincident particles
      s += r2 > 0.0 ? cc * fp / r * t : 0.0;
      const double cf = cc * f;
      gx += cf * ux; gy += cf * uy; gz += cf * uz;
      gh -= cc * t * (5.0 * f + r * fp) * inv_h;  // dF/dh = -(5 F + r F')/h
    }
    gx += s * dx; gy += s * dy; gz += s * dz;
  }
  const int64_t k = id[i];
  if (accumulate) {
    qbar[3 * k] += gx; qbar[3 * k + 1] += gy; qbar[3 * k + 2] += gz;
  } else {
    qbar[3 * k] = gx; qbar[3 * k + 1] = gy; qbar[3 * k + 2] = gz;
  }
  // self term of rho_i: m dW/dh(0) = -3 m W(0)/h
  thbar[3 * k] += 0.5 * gh - 3.0 * m * c.W0 * inv_h * vi.w;
}

__global__ void k_adj_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

// Column sums of x[n][ncols] (ncols <= 3) in a fixed order: per-block
// partials, then one block.
constexpr int kSumBlocks = 256;

__global__ void __launch_bounds__(256) k_adj_sum_partial(const double* __restrict__ x, int64_t n, int ncols,
                                                         double* __restrict__ partial) {
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < ncols; ++k) s[k] += x[i * ncols + k];
  __shared__ double red[3][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < ncols; ++k) {
    double v = s[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[k][wid] = v;
  }
  __syncthreads();
  if (wid == 0)
    for (int k = 0; k < ncols; ++k) {
      double v = lane < 8 ? red[k][lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) partial[blockIdx.x * 3 + k] = v;
    }
}

__global__ void k_adj_sum_final(const double* __restrict__ partial, int nb, int ncols, double* __restrict__ out) {
  const int lane = threadIdx.x;
  for (int k = 0; k < ncols; ++k) {
    double v = 0.0;
    for (int b = lane; b < nb; b += 32) v += partial[b * 3 + k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) out[k] = v;
  }
}

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_adj_gather(const Consts& c, const Workspace& w, int cur, const double* pbar_id, double scale, D4* vs4,
                       cudaStream_t s) {
  if (c.N == 0) return;
  k_adj_gather<<<nblocks(c.N, 256), 256, 0, s>>>(c.N, w.id[cur], pbar_id, scale, vs4);
}

void launch_adj_pairsum(const Consts& c, const Workspace& w, int cur, int mode, const D4* vs4, double* A,
                        cudaStream_t s) {
  if (c.N == 0) return;
  const D4* qp4 = (const D4*)w.qp4;
  const D4* q4 = (const D4*)w.q4[cur];
  const unsigned nb = nblocks(c.N, 128);
  if (c.kernel == SDPD_KERNEL_LUCY) {
    if (mode == 0) k_adj_pairsum<SDPD_KERNEL_LUCY, 0><<<nb, 128, 0, s>>>(c, qp4, q4, vs4, w.nlist, w.nn, A, w.status);
    else k_adj_pairsum<SDPD_KERNEL_LUCY, 1><<<nb, 128, 0, s>>>(c, qp4, q4, vs4, w.nlist, w.nn, A, w.status);
  } else {
    if (mode == 0) k_adj_pairsum<SDPD_KERNEL_CUBIC, 0><<<nb, 128, 0, s>>>(c, qp4, q4, vs4, w.nlist, w.nn, A, w.status);
    else k_adj_pairsum<SDPD_KERNEL_CUBIC, 1><<<nb, 128, 0, s>>>(c, qp4, q4, vs4, w.nlist, w.nn, A, w.status);
  }
}

void launch_adj_mid_step(const Consts& c, const Workspace& w, int cur, const double* A, bool kick1, bool kick2,
                         const double* deps_prev, double* Sbar_cur, double* Sbar_prev, const double* epsbar_n,
                         double* epsbar0, D4* vs4, double* thbar, cudaStream_t s) {
  if (c.N == 0) return;
  const int flags = (kick1 ? kAdjKick1 : 0) | (kick2 ? kAdjKick2 : 0);
  k_adj_mid_step<<<nblocks(c.N, 256), 256, 0, s>>>(c, (D4*)w.qp4, (const double*)w.rho[cur], w.eps[cur], w.id[cur],
                                                    A, flags, deps_prev, Sbar_cur, Sbar_prev, epsbar_n, epsbar0,
                                                    vs4, thbar);
}

void launch_adj_freeze(const Consts& c, const Workspace& w, int cur, const double* pre, double* dp, double* de,
                       cudaStream_t s) {
  if (c.N == 0) return;
  k_adj_freeze<<<nblocks(c.N, 256), 256, 0, s>>>(c.N, c.c_rho / (c.C_K * c.m), w.id[cur], (double*)w.px[cur],
                                                  (double*)w.py[cur], (double*)w.pz[cur], w.eps[cur],
                                                  (const double*)w.rho[cur], (D4*)w.qp4, pre, dp, de);
}

void launch_adj_increment(const Consts& c, const Workspace& w, int cur, const double* dp, const double* de,
                          cudaStream_t s) {
  if (c.N == 0) return;
  k_adj_increment<<<nblocks(c.N, 256), 256, 0, s>>>(c.N, c.c_rho / (c.C_K * c.m), w.id[cur], (double*)w.px[cur],
                                                     (double*)w.py[cur], (double*)w.pz[cur], w.eps[cur],
                                                     (const double*)w.rho[cur], (D4*)w.qp4, dp, de);
}

void launch_adj_mid_virial(const Consts& c, const Workspace& w, int cur, const double* A, double wt, D4* vs4,
                           double* val_id, double* gp, double* geps, double* thbar, cudaStream_t s) {
  if (c.N == 0) return;
  k_adj_mid_virial<<<nblocks(c.N, 256), 256, 0, s>>>(
      c, (const D4*)w.qp4, (const double*)w.rho[cur], w.eps[cur], (const double*)w.px[cur],
      (const double*)w.py[cur], (const double*)w.pz[cur], w.id[cur], A, wt, vs4, val_id, gp, geps, thbar);
}

void launch_adj_back(const Consts& c, const Workspace& w, int cur, int mode, double wt, const D4* vs4,
                     int accumulate, double* qbar, double* thbar, cudaStream_t s) {
  if (c.N == 0) return;
  const D4* qp4 = (const D4*)w.qp4;
  const D4* q4 = (const D4*)w.q4[cur];
  const unsigned nb = nblocks(c.N, 128);
  const int32_t* id = w.id[cur];
#define SDPD_ADJ_BACK(KIND, MODE) \
  k_adj_back<KIND, MODE><<<nb, 128, 0, s>>>(c, qp4, q4, vs4, id, w.nlist, w.nn, wt, accumulate, qbar, thbar, w.status)
  if (c.kernel == SDPD_KERNEL_LUCY) {
    if (mode == 0) SDPD_ADJ_BACK(SDPD_KERNEL_LUCY, 0);
    else if (mode == 1) SDPD_ADJ_BACK(SDPD_KERNEL_LUCY, 1);
    else SDPD_ADJ_BACK(SDPD_KERNEL_LUCY, 2);
  } else {
    if (mode == 0) SDPD_ADJ_BACK(SDPD_KERNEL_CUBIC, 0);
    else if (mode == 1) SDPD_ADJ_BACK(SDPD_KERNEL_CUBIC, 1);
    else SDPD_ADJ_BACK(SDPD_KERNEL_CUBIC, 2);
  }
#undef SDPD_ADJ_BACK
}

void launch_adj_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  if (n == 0) return;
  k_adj_axpy<<<nblocks(n, 256), 256, 0, s>>>(n, a, x, y);
}

size_t adj_sum_partial_doubles() { return (size_t)kSumBlocks * 3; }

void launch_adj_sum(const double* x, int64_t n, int ncols, double* partial, double* out, cudaStream_t s) {
  k_adj_sum_partial<<<kSumBlocks, 256, 0, s>>>(x, n, ncols, partial);
  k_adj_sum_final<<<1, 32, 0, s>>>(partial, kSumBlocks, ncols, out);
}

}  // namespace sdpd
