// sdpd_pair.cu -- the two pair passes of Velocity Verlet: the density sum of
// Eq. (sdpd-rho-v) with the equation-of-state update of Section 3.1, and the
// conservative force of Eq. (cons-forces) with the half kick (and, for the
// first kick of a step, the drift and the cell binning of the new position).
//
// One thread per particle in storage order; the neighbour search walks the
// 27 cells around the particle's cell (cell side >= h) with the predicate
// r^2 < h^2 after the periodic minimum image.
#include "sdpd_internal.cuh"

namespace sdpd {

// Geometry of one home particle: displacement to a neighbour j.
// Float64: absolute coordinates and the minimum image.
// Mixed: coordinates relative to the own cell's lower corner; per axis and
// neighbour offset o in {-1, 0, +1} the home coordinate shifted by the
// (exact, fixed-point) distance between the two cells' corners.
template <class P>
struct Home;

template <>
struct Home<Fp64> {
  double x, y, z;
  int cx, cy, cz;
  double mx, my, mz, px_, py_, pz_;  // image shifts of the neighbour offsets -1 and +1 per axis
  double fx, fy, fz;                 // shifts of the current neighbour cell
  __device__ void init(const Consts& c, const D4& q, int cx_, int cy_, int cz_, const uint32_t*, const uint32_t*,
                       const uint32_t*) {
    x = q.x; y = q.y; z = q.z;
    cx = cx_; cy = cy_; cz = cz_;
    mx = image_shift(cx, -1, c.nc[0], c.L[0]); px_ = image_shift(cx, 1, c.nc[0], c.L[0]);
    my = image_shift(cy, -1, c.nc[1], c.L[1]); py_ = image_shift(cy, 1, c.nc[1], c.L[1]);
    mz = image_shift(cz, -1, c.nc[2], c.L[2]); pz_ = image_shift(cz, 1, c.nc[2], c.L[2]);
    fx = fy = fz = 0.0;
  }
  // neighbour cell (nx, ny, nz) = (cx + ox, ...) wrapped: its image shifts
  __device__ __forceinline__ void frame(int nx, int ny, int nz) {
    fx = nx - cx > 1 ? mx : (nx - cx < -1 ? px_ : 0.0);
    fy = ny - cy > 1 ? my : (ny - cy < -1 ? py_ : 0.0);
    fz = nz - cz > 1 ? mz : (nz - cz < -1 ? pz_ : 0.0);
  }
  __device__ __forceinline__ void frames_all(const Consts&) {}
  __device__ __forceinline__ static double pick(uint32_t k, double m, double p) {
    return k == 0 ? m : (k == 2 ? p : 0.0);
  }
  __device__ __forceinline__ void disp_code(uint32_t code, const D4& qj, double& dx, double& dy, double& dz) const {
    const double sx = pick(code & 3u, mx, px_), sy = pick((code >> 2) & 3u, my, py_),
                 sz = pick((code >> 4) & 3u, mz, pz_);
    dx = __dsub_rn(x, qj.x);
    dy = __dsub_rn(y, qj.y);
    dz = __dsub_rn(z, qj.z);
    if (sx != 0.0) dx = __dadd_rn(dx, sx);
    if (sy != 0.0) dy = __dadd_rn(dy, sy);
    if (sz != 0.0) dz = __dadd_rn(dz, sz);
  }
  __device__ __forceinline__ void disp(const D4& qj, double& dx, double& dy, double& dz) const {
    dx = __dsub_rn(x, qj.x);
    dy = __dsub_rn(y, qj.y);
    dz = __dsub_rn(z, qj.z);
    if (fx != 0.0) dx = __dadd_rn(dx, fx);
    if (fy != 0.0) dy = __dadd_rn(dy, fy);
    if (fz != 0.0) dz = __dadd_rn(dz, fz);
  }
};

template <>
struct Home<Mixed> {
  float x, y, z, sx, sy, sz;
  int cx, cy, cz;
  const uint32_t *xmx, *xmy, *xmz;
  float hx, hy, hz;  // home coordinates in the frame of the current neighbour cell
  __device__ void init(const Consts& c, const F4& q, int cx_, int cy_, int cz_, const uint32_t* xmx_,
                       const uint32_t* xmy_, const uint32_t* xmz_) {
    x = q.x; y = q.y; z = q.z;
    sx = (float)c.scale[0]; sy = (float)c.scale[1]; sz = (float)c.scale[2];
    cx = cx_; cy = cy_; cz = cz_;
    xmx = xmx_; xmy = xmy_; xmz = xmz_;
  }
  // shift into the frame of neighbour cell (nx, ny, nz): exact fixed-point
  // distance between the two cells' lower corners
  __device__ __forceinline__ void frame(int nx, int ny, int nz) {
    hx = x + (float)(int32_t)(__ldg(&xmx[cx]) - __ldg(&xmx[nx])) * sx;
    hy = y + (float)(int32_t)(__ldg(&xmy[cy]) - __ldg(&xmy[ny])) * sy;
    hz = z + (float)(int32_t)(__ldg(&xmz[cz]) - __ldg(&xmz[nz])) * sz;
  }
  __device__ __forceinline__ void disp(const F4& qj, float& dx, float& dy, float& dz) const {
    dx = hx - qj.x;
    dy = hy - qj.y;
    dz = hz - qj.z;
  }
  // all nine shifted home coordinates, for walking a neighbour list
  float fx[3], fy[3], fz[3];
  __device__ __forceinline__ void frames_all(const Consts& c) {
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      int nx = cx + o - 1, ny = cy + o - 1, nz = cz + o - 1;
      nx += nx < 0 ? c.nc[0] : (nx >= c.nc[0] ? -c.nc[0] : 0);
      ny += ny < 0 ? c.nc[1] : (ny >= c.nc[1] ? -c.nc[1] : 0);
      nz += nz < 0 ? c.nc[2] : (nz >= c.nc[2] ? -c.nc[2] : 0);
      frame(nx, ny, nz);
      fx[o] = hx; fy[o] = hy; fz[o] = hz;
    }
  }
  __device__ __forceinline__ static float pick(const float* v, uint32_t k) {
    return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]);
  }
  __device__ __forceinline__ void disp_code(uint32_t code, const F4& qj, float& dx, float& dy, float& dz) const {
    dx = pick(fx, code & 3u) - qj.x;
    dy = pick(fy, (code >> 2) & 3u) - qj.y;
    dz = pick(fz, (code >> 4) & 3u) - qj.z;
  }
};

__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// ---------------------------------------------------------------------------
// Density, Eq. (sdpd-rho-v): rho_i = m W(0) + sum_{j != i, r_ij < h} m W(r_ij);
// then the energies at fixed entropy (Section 3.1): S_i = S(eps_i, rho_old),
// eps_i = E(S_i, rho_i), and pi_i = P_i / rho_i^2 from Eq. (pg-eos):
// P = c_rho rho eps / (C_K m).
// ---------------------------------------------------------------------------
template <class P, int KIND>
__global__ void __launch_bounds__(128, P::mixed ? 12 : 1) k_density(Consts c, Arrays<P> a, typename P::V4* __restrict__ qp4,
                                                 const int32_t* __restrict__ cell_start,
                                                 const int32_t* __restrict__ mrank,
                                                 const uint32_t* __restrict__ xmx,
                                                 const uint32_t* __restrict__ xmy,
                                                 const uint32_t* __restrict__ xmz, int update_eos,
                                                 int32_t* __restrict__ ncount_by_id,
                                                 uint32_t* __restrict__ nlist, int32_t* __restrict__ nn,
                                                 int32_t* __restrict__ ovf_list, int32_t* __restrict__ ovf_count,
                                                 int32_t* __restrict__ ovf_other, const float4* __restrict__ qf4,
                                                 typename P::V4* __restrict__ qr4, uint32_t* __restrict__ cend) {
  using R = typename P::R;
  using V4 = typename P::V4;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0) *ovf_other = 0;  // the other slot: its readers have run
  if (i >= c.N) return;
  const V4 qi = ld4(&a.q4[i]);
  float4 fi = make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (!P::mixed) fi = qf4[i];
  int cx, cy, cz;
  unpack_cell(w_to_cellbits(qi.w), cx, cy, cz);
  Home<P> home;
  home.init(c, qi, cx, cy, cz, xmx, xmy, xmz);
  const R h2 = (R)c.h2, inv_h = R(1) / (R)c.h, cW = (R)c.cW;
  R acc = R(0);
  int cnt = 0;
  uint32_t* wp = nlist + nbr_slot(i, 0, c.nbr_cap);  // where entry cnt of the list goes
  // Every lane walks the 27 cells in the same order (z, then y, then x
  // offset, each -1, 0, +1), so the warp's loops stay converged.  Per row
  // (oz, oy) of three cells, cend[row][i] records where the list stands:
  // byte 0 at the row's start, byte 1 + k after its k-th cell (counts
  // clamped to 255).  The sweep's schedule finds each block's pairs in
  // these cell runs of the list.
#pragma unroll 1
  for (int oz = -1; oz <= 1; ++oz) {
    const int nz = wrapc(cz + oz, c.nc[2]);
#pragma unroll 1
    for (int oy = -1; oy <= 1; ++oy) {
      const int ny = wrapc(cy + oy, c.nc[1]);
      uint32_t rw = (uint32_t)min(cnt, 255);
#pragma unroll 1
      for (int ox = -1; ox <= 1; ++ox) {
        const int nx = wrapc(cx + ox, c.nc[0]);
        const int r = __ldg(&mrank[nx + c.nc[0] * (ny + c.nc[1] * nz)]);
        const int beg = __ldg(&cell_start[r]), end = __ldg(&cell_start[r + 1]);
        home.frame(nx, ny, nz);
        const uint32_t code = nbr_entry(0, ox, oy, oz);
#pragma unroll 4
        for (int j = beg; j < end; ++j) {
          if constexpr (!P::mixed) {  // float32 pre-test: skips only pairs with r >= h
            if (j == i) continue;
            const float4 fj = __ldg(&qf4[j]);
            float ex = fi.x - fj.x, ey = fi.y - fj.y, ez = fi.z - fj.z;
            ex = ex > c.halfLf[0] ? ex - c.Lf[0] : (ex < -c.halfLf[0] ? ex + c.Lf[0] : ex);
            ey = ey > c.halfLf[1] ? ey - c.Lf[1] : (ey < -c.halfLf[1] ? ey + c.Lf[1] : ey);
            ez = ez > c.halfLf[2] ? ez - c.Lf[2] : (ez < -c.halfLf[2] ? ez + c.Lf[2] : ez);
            if (ex * ex + ey * ey + ez * ez >= c.h2_filter) continue;
          }
          const V4 qj = ld4(&a.q4[j]);
          R dx, dy, dz;
          home.disp(qj, dx, dy, dz);
          const R r2 = r2_of(dx, dy, dz);
          // kept neighbours (about one candidate in six) take the short
          // branch: the kernel value and one list store at a stepped address
          if (r2 < h2 && j != i) {
            acc += kernel_W<KIND>(pair_r(r2) * inv_h, cW);
            if (cnt < c.nbr_cap) *wp = ((uint32_t)j << 6) | code;
            wp += (cnt & 3) == 3 ? 125 : 1;  // nbr_slot(i, cnt + 1) - nbr_slot(i, cnt)
            ++cnt;
          }
        }
        rw |= (uint32_t)min(cnt, 255) << (8 * (ox + 2));
      }
      cend[(int64_t)((oz + 1) * 3 + (oy + 1)) * c.N + i] = rw;
    }
  }
  if (ncount_by_id) ncount_by_id[a.id[i]] = cnt;
  nn[i] = cnt;
  if (cnt > c.nbr_cap) ovf_list[atomicAdd(ovf_count, 1)] = (int32_t)i;  // forces from the cells
  const R rho_new = (R)c.m * ((R)c.W0 + acc);
  double e = a.eps[i];
  if (update_eos) {
    if constexpr (P::mixed) {
      // eps * (rho_new / rho_old)^(c_rho / C_K), the factor minus one formed
      // from log1p / expm1 of small arguments so float32 keeps it accurate
      const float ro = a.rho[i];
      const float g = expm1f((float)(c.c_rho / c.C_K) * log1pf((rho_new - ro) / ro));
      e = fma(e, (double)g, e);
    } else {
      const double S = c.C_K * log(e) - c.c_rho * log((double)a.rho[i]);
      e = exp((S + c.c_rho * log((double)rho_new)) / c.C_K);
    }
    a.eps[i] = e;
  }
  a.rho[i] = rho_new;
  R pi;
  if constexpr (P::mixed) pi = (float)e * (float)(c.c_rho / (c.C_K * c.m)) / rho_new;
  else pi = e * (c.c_rho / (c.C_K * c.m)) / rho_new;
  V4 o = qi;
  o.w = pi;
  st4(&qp4[i], o);
  o.w = rho_new;  // positions and density together for the sweep's pair geometry
  st4(&qr4[i], o);
}

// Kick (and, with dt_drift != 0, drift and binning) of particle i with the
// force sum f (before the factor m^2): p_i += m^2 f dt/2 of Eq. (sdpd-verlet),
// q_i += p_i dt/m wrapped, and the new cell counted for the sort.
template <class P>
__device__ __forceinline__ void kick_particle(const Consts& c, const Arrays<P>& a, int64_t i, typename P::R fx,
                                              typename P::R fy, typename P::R fz, double half_dt, double dt_drift,
                                              typename P::Q* __restrict__ qdx, typename P::Q* __restrict__ qdy,
                                              typename P::Q* __restrict__ qdz, int32_t* __restrict__ key,
                                              int32_t* __restrict__ slot, int32_t* __restrict__ cell_count,
                                              const int32_t* __restrict__ mrank, double* __restrict__ force_by_id,
                                              const float drift_f[3]) {
  using R = typename P::R;
  const R m2 = (R)(c.m * c.m);
  fx *= m2; fy *= m2; fz *= m2;
  if (force_by_id) {
    const int64_t k = a.id[i];
    force_by_id[3 * k] = fx;
    force_by_id[3 * k + 1] = fy;
    force_by_id[3 * k + 2] = fz;
  }
  const R hdt = (R)half_dt;  // one conversion per thread
  R px = a.px[i] + fx * hdt, py = a.py[i] + fy * hdt, pz = a.pz[i] + fz * hdt;
  a.px[i] = px; a.py[i] = py; a.pz[i] = pz;
  if (dt_drift != 0.0) {
    int nc3[3];
    if constexpr (P::mixed) {
      // fixed point: the displacement in units of L / 2^32, wrap-around = periodic
      uint32_t ux = a.qx[i] + (uint32_t)__float2int_rn(px * drift_f[0]);
      uint32_t uy = a.qy[i] + (uint32_t)__float2int_rn(py * drift_f[1]);
      uint32_t uz = a.qz[i] + (uint32_t)__float2int_rn(pz * drift_f[2]);
      qdx[i] = ux; qdy[i] = uy; qdz[i] = uz;
      nc3[0] = (int)__umulhi(ux, (uint32_t)c.nc[0]);
      nc3[1] = (int)__umulhi(uy, (uint32_t)c.nc[1]);
      nc3[2] = (int)__umulhi(uz, (uint32_t)c.nc[2]);
    } else {
      double pp[3] = {px, py, pz}, qq[3] = {a.qx[i], a.qy[i], a.qz[i]};
      for (int d = 0; d < 3; ++d) {
        double x = __dadd_rn(qq[d], __ddiv_rn(__dmul_rn(pp[d], dt_drift), c.m));
        if (x >= c.L[d]) x = __dsub_rn(x, c.L[d]);
        else if (x < 0.0) x = __dadd_rn(x, c.L[d]);
        if (x >= c.L[d]) x = 0.0;
        qq[d] = x;
        int cc = (int)floor(__ddiv_rn(x, c.cs[d]));
        nc3[d] = cc >= c.nc[d] ? c.nc[d] - 1 : (cc < 0 ? 0 : cc);
      }
      qdx[i] = qq[0]; qdy[i] = qq[1]; qdz[i] = qq[2];
    }
    const int r = mrank[nc3[0] + c.nc[0] * (nc3[1] + c.nc[1] * nc3[2])];
    key[i] = r;
    slot[i] = atomicAdd(&cell_count[r], 1);
  }
}

// Force and kick of a particle with more neighbours than its list row
// holds: the pair force sum from the 27 cells around it, with the
// candidates, the predicate and the order of the density pass, so that the
// sum is the one a long enough list would give.
template <class P, int KIND>
__device__ __forceinline__ void force_from_cells(const Consts& c, const Arrays<P>& a, int64_t i,
                                              const typename P::V4* __restrict__ qp4,
                                              const int32_t* __restrict__ cell_start,
                                              const int32_t* __restrict__ mrank, const uint32_t* xmx,
                                              const uint32_t* xmy, const uint32_t* xmz, double half_dt,
                                              double dt_drift, typename P::Q* qdx, typename P::Q* qdy,
                                              typename P::Q* qdz, int32_t* key, int32_t* slot,
                                              int32_t* cell_count, double* force_by_id, float3 drift3) {
  using R = typename P::R;
  using V4 = typename P::V4;
  const V4 qi = ld4(&qp4[i]);
  int cx, cy, cz;
  unpack_cell(w_to_cellbits(ld4(&a.q4[i]).w), cx, cy, cz);
  Home<P> home;
  home.init(c, qi, cx, cy, cz, xmx, xmy, xmz);
  const R h2 = (R)c.h2, inv_h = R(1) / (R)c.h, cF = (R)c.cF;
  R fx = R(0), fy = R(0), fz = R(0);
  for (int oz = -1; oz <= 1; ++oz) {
    const int nz = wrapc(cz + oz, c.nc[2]);
    for (int oy = -1; oy <= 1; ++oy) {
      const int ny = wrapc(cy + oy, c.nc[1]);
      for (int ox = -1; ox <= 1; ++ox) {
        const int nx = wrapc(cx + ox, c.nc[0]);
        const int r = __ldg(&mrank[nx + c.nc[0] * (ny + c.nc[1] * nz)]);
        const int beg = __ldg(&cell_start[r]), end = __ldg(&cell_start[r + 1]);
        home.frame(nx, ny, nz);
        for (int j = beg; j < end; ++j) {
          if (j == i) continue;
          const V4 qj = ld4(&qp4[j]);
          R dx, dy, dz;
          home.disp(qj, dx, dy, dz);
          const R r2 = r2_of(dx, dy, dz);
          if (r2 < h2) {
            const R s = (qi.w + qj.w) * kernel_F<KIND>(pair_r(r2) * inv_h, cF);
            fx += s * dx;
            fy += s * dy;
            fz += s * dz;
          }
        }
      }
    }
  }
  const float drift_f[3] = {drift3.x, drift3.y, drift3.z};
  kick_particle<P>(c, a, i, fx, fy, fz, half_dt, dt_drift, qdx, qdy, qdz, key, slot, cell_count, mrank,
                   force_by_id, drift_f);
}

// ---------------------------------------------------------------------------
// Conservative force, Eq. (cons-forces): F_i = sum_{j != i, r_ij < h}
// m^2 (pi_i + pi_j) F(r_ij) r_ij, and the kick p_i += F_i dt/2 of Eq.
// (sdpd-verlet).  With drift: q_i += p_i dt/m (wrapped), new cell counted
// for the sort.  A particle whose neighbour list overflowed its row (listed
// by the density pass) is left to k_force_overflow.
// ---------------------------------------------------------------------------
template <class P, int KIND>
__global__ void __launch_bounds__(128, P::mixed ? (KIND == SDPD_KERNEL_LUCY ? 16 : 12) : 1) k_force(Consts c, Arrays<P> a, const typename P::V4* __restrict__ qp4,
                                               const int32_t* __restrict__ cell_start,
                                               const int32_t* __restrict__ mrank,
                                               const uint32_t* __restrict__ xmx,
                                               const uint32_t* __restrict__ xmy,
                                               const uint32_t* __restrict__ xmz, double half_dt,
                                               double dt_drift, typename P::Q* __restrict__ qdx,
                                               typename P::Q* __restrict__ qdy,
                                               typename P::Q* __restrict__ qdz, int32_t* __restrict__ key,
                                               int32_t* __restrict__ slot, int32_t* __restrict__ cell_count,
                                               double* __restrict__ force_by_id,
                                               const uint32_t* __restrict__ nlist, const int32_t* __restrict__ nn,
                                               float3 drift3) {
  // mixed path: dt / m * 2^32 / L per axis, computed on the host
  const float drift_f[3] = {drift3.x, drift3.y, drift3.z};
  using R = typename P::R;
  using V4 = typename P::V4;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int n = i < c.N ? nn[i] : 0;
  if (i < c.N && n <= c.nbr_cap) {
    const V4 qi = ld4(&a.q4[i]);
    const R pi_i = ld4(&qp4[i]).w;
    int cx, cy, cz;
    unpack_cell(w_to_cellbits(qi.w), cx, cy, cz);
    Home<P> home;
    home.init(c, qi, cx, cy, cz, xmx, xmy, xmz);
    const R inv_h = R(1) / (R)c.h, cF = (R)c.cF;
    R fx = R(0), fy = R(0), fz = R(0);
    home.frames_all(c);
    // four entries per 16-byte load (a warp's loads are contiguous, see
    // nbr_slot), then four independent neighbour gathers
    for (int k = 0; k < n; k += 4) {
      const uint4 e4 = __ldg(reinterpret_cast<const uint4*>(nlist + nbr_slot(i, k, c.nbr_cap)));
      const uint32_t ev[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (k + u < n) {
          const uint32_t e = ev[u];
          const V4 qj = ld4(&qp4[e >> 6]);
          R dx, dy, dz;
          home.disp_code(e & 63u, qj, dx, dy, dz);
          const R r2 = r2_of(dx, dy, dz);
          const R s = (pi_i + qj.w) * kernel_F<KIND>(pair_r(r2) * inv_h, cF);
          fx += s * dx;
          fy += s * dy;
          fz += s * dz;
        }
      }
    }
    kick_particle<P>(c, a, i, fx, fy, fz, half_dt, dt_drift, qdx, qdy, qdz, key, slot, cell_count, mrank,
                     force_by_id, drift_f);
  }
}

// The particles that k_force left: more neighbours than a list row holds.
// A few thread blocks loop over the density pass's overflow list (usually
// empty: the launch then ends at once).
constexpr int kOverflowBlocks = 4;
template <class P, int KIND>
__global__ void __launch_bounds__(128) k_force_overflow(Consts c, Arrays<P> a, const typename P::V4* __restrict__ qp4,
                                                        const int32_t* __restrict__ cell_start,
                                                        const int32_t* __restrict__ mrank,
                                                        const uint32_t* __restrict__ xmx,
                                                        const uint32_t* __restrict__ xmy,
                                                        const uint32_t* __restrict__ xmz, double half_dt,
                                                        double dt_drift, typename P::Q* __restrict__ qdx,
                                                        typename P::Q* __restrict__ qdy,
                                                        typename P::Q* __restrict__ qdz, int32_t* __restrict__ key,
                                                        int32_t* __restrict__ slot, int32_t* __restrict__ cell_count,
                                                        double* __restrict__ force_by_id, float3 drift3,
                                                        const int32_t* __restrict__ ovf_list,
                                                        const int32_t* __restrict__ ovf_count) {
  const int novf = *ovf_count;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < novf; q += gridDim.x * blockDim.x)
    force_from_cells<P, KIND>(c, a, ovf_list[q], qp4, cell_start, mrank, xmx, xmy, xmz, half_dt, dt_drift, qdx, qdy,
                              qdz, key, slot, cell_count, force_by_id, drift3);
}

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// threads per block of the pair passes (one thread per particle, no shared
// memory, so any of the accepted sizes gives the same results)
static inline int pair_block(const Consts& c) { return pair_threads_ok(c.pair_threads) ? c.pair_threads : 128; }

template <class P>
void launch_density(const Consts& c, const Workspace& w, int cur, int update_eos, int32_t* ncount_by_id,
                    cudaStream_t s) {
  if (c.N == 0) return;
  Arrays<P> a = view<P>(w, cur);
  auto qp4 = (typename P::V4*)w.qp4;
  const int t = pair_block(c);
  const int sl = (*w.ovf_slot ^= 1);  // this pass's slot of the overflow list
  int32_t* ovf_list = w.ovf_list + (size_t)sl * (size_t)c.N;
  int32_t* ovf_count = w.ovf_count + sl;
  int32_t* ovf_other = w.ovf_count + (sl ^ 1);
  if (c.kernel == SDPD_KERNEL_LUCY)
    k_density<P, SDPD_KERNEL_LUCY><<<blocks_for(c.N, t), t, 0, s>>>(
        c, a, qp4, w.cell_start, w.mrank, w.xmin[0], w.xmin[1], w.xmin[2], update_eos, ncount_by_id, w.nlist,
        w.nn, ovf_list, ovf_count, ovf_other, w.qf4, (typename P::V4*)w.qr4, w.cend);
  else
    k_density<P, SDPD_KERNEL_CUBIC><<<blocks_for(c.N, t), t, 0, s>>>(
        c, a, qp4, w.cell_start, w.mrank, w.xmin[0], w.xmin[1], w.xmin[2], update_eos, ncount_by_id, w.nlist,
        w.nn, ovf_list, ovf_count, ovf_other, w.qf4, (typename P::V4*)w.qr4, w.cend);
}

template <class P>
void launch_force(const Consts& c, const Workspace& w, int cur, double half_dt, double dt_drift,
                  double* force_by_id, cudaStream_t s) {
  if (c.N == 0) return;
  Arrays<P> a = view<P>(w, cur);
  auto qp4 = (const typename P::V4*)w.qp4;
  auto qdx = (typename P::Q*)w.qdx;
  auto qdy = (typename P::Q*)w.qdy;
  auto qdz = (typename P::Q*)w.qdz;
  const float3 drift3 = make_float3((float)(dt_drift / c.m * c.inv_scale[0]), (float)(dt_drift / c.m * c.inv_scale[1]),
                                    (float)(dt_drift / c.m * c.inv_scale[2]));
  const int sl = *w.ovf_slot;  // the overflow list of the latest density pass
  const int32_t* ovf_list = w.ovf_list + (size_t)sl * (size_t)c.N;
  const int32_t* ovf_count = w.ovf_count + sl;
  const int t = pair_block(c);
  if (c.kernel == SDPD_KERNEL_LUCY) {
    k_force<P, SDPD_KERNEL_LUCY><<<blocks_for(c.N, t), t, 0, s>>>(
        c, a, qp4, w.cell_start, w.mrank, w.xmin[0], w.xmin[1], w.xmin[2], half_dt, dt_drift, qdx, qdy,
        qdz, w.key, w.slot, w.cell_count, force_by_id, w.nlist, w.nn, drift3);
    k_force_overflow<P, SDPD_KERNEL_LUCY><<<kOverflowBlocks, 128, 0, s>>>(
        c, a, qp4, w.cell_start, w.mrank, w.xmin[0], w.xmin[1], w.xmin[2], half_dt, dt_drift, qdx, qdy,
        qdz, w.key, w.slot, w.cell_count, force_by_id, drift3, ovf_list, ovf_count);
  } else {
    k_force<P, SDPD_KERNEL_CUBIC><<<blocks_for(c.N, t), t, 0, s>>>(
        c, a, qp4, w.cell_start, w.mrank, w.xmin[0], w.xmin[1], w.xmin[2], half_dt, dt_drift, qdx, qdy,
        qdz, w.key, w.slot, w.cell_count, force_by_id, w.nlist, w.nn, drift3);
    k_force_overflow<P, SDPD_KERNEL_CUBIC><<<kOverflowBlocks, 128, 0, s>>>(
        c, a, qp4, w.cell_start, w.mrank, w.xmin[0], w.xmin[1], w.xmin[2], half_dt, dt_drift, qdx, qdy,
        qdz, w.key, w.slot, w.cell_count, force_by_id, drift3, ovf_list, ovf_count);
  }
}

template void launch_density<Fp64>(const Consts&, const Workspace&, int, int, int32_t*, cudaStream_t);
template void launch_density<Mixed>(const Consts&, const Workspace&, int, int, int32_t*, cudaStream_t);
template void launch_force<Fp64>(const Consts&, const Workspace&, int, double, double, double*,
                                 cudaStream_t);
template void launch_force<Mixed>(const Consts&, const Workspace&, int, double, double, double*,
                                  cudaStream_t);

}  // namespace sdpd
