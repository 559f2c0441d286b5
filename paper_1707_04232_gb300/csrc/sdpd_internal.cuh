// sdpd_internal.cuh -- device building blocks and the handle layout shared by
// the translation units of the SDPD library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sdpd.h"

namespace sdpd {

// ---------------------------------------------------------------------------
// Capacities of one 2x2x2 block of cells (the unit of the pair colouring).
// ---------------------------------------------------------------------------
constexpr int kMaxBlock = 256;   // particles in a block (8-bit local index)
constexpr int kMaxPairs = 2048;  // owned pairs of a block
constexpr int kMaxLevels = 255;  // dependency levels of a block's pair schedule
// Schedule header of a block beyond one of these capacities: its sweep runs
// in canonical order, one pair after the other, on the whole warp that takes
// it (no shared-memory schedule), so any block size completes.
constexpr uint32_t kHdrBig = 0xFFFFFFFFu;

// Sticky device status bits, mapped to SDPD_ERR_* on the host.
enum : int {
  kStNegative = 1,    // SSA produced eps <= 0
  kStNaN = 2,         // non-finite momentum / energy
  kStCapacity = 4,    // a capacity that has no fallback was exceeded
  kStBadEnergy = 8,   // set_state got eps <= 0
  kStNbrCap = 16,     // a gradient pass met a neighbour list longer than its row
};

// Per-run constants; every kernel gets a copy by value.
struct Consts {
  int64_t N;
  int nc[3];
  int ncell;
  double L[3], halfL[3], cs[3];
  double scale[3];      // mixed precision: box side / 2^32 (fixed-point unit)
  double inv_scale[3];  // 2^32 / box side
  double h, h2, m, kB;
  double C_K, c_rho;
  double kpar_m2, kperp_m2;  // (10/3 eta + 4 zeta) m^2 and (5/3 eta - zeta) m^2
  double cW, cF, W0;         // kernel constants and W(0)
  int kernel, scheme;
  int nbr_cap;               // neighbour-list entries per particle
  // float64 path: float32 pre-test of the neighbour predicate.  A candidate
  // whose float32 r^2 (from float32 copies of the positions) is >= h2_filter
  // has r^2 >= h^2 in float64 (bound on the conversion and rounding errors
  // set on the host), so it is skipped without float64 arithmetic.
  float Lf[3], halfLf[3], h2_filter;
  // launch shapes (results do not depend on them): the block schedule of the
  // sweep's colour launches and the threads per block of the pair passes
  int fd_variant, pair_threads;
};

// Block schedules of the colour kernel (see launch_fd_colours) and the
// thread-block sizes the pair passes accept.
constexpr int kFdVariants = 5;
__host__ __device__ constexpr int fd_default_variant(bool mixed) { return mixed ? 0 : 1; }
__host__ __device__ constexpr bool pair_threads_ok(int t) { return t == 32 || t == 64 || t == 128; }
// whether a block schedule's shared memory fits a thread block (float64
// blocks take twice the bytes of mixed ones)
bool fd_variant_fits(bool mixed, int v);

// Neighbour-list entry: neighbour index << 6 | stencil offset code, the code
// holding (o + 1) per axis in 2 bits (x lowest) for o in {-1, 0, +1}.
__host__ __device__ __forceinline__ uint32_t nbr_entry(int j, int ox, int oy, int oz) {
  return ((uint32_t)j << 6) | (uint32_t)((ox + 1) | ((oy + 1) << 2) | ((oz + 1) << 4));
}

// Position of entry k of particle i's neighbour list (cap entries, a multiple
// of 4, per particle).  The lists of 32 consecutive particles (one warp of a
// pair pass) are interleaved in groups of four entries:
// [i / 32][k / 4][i % 32][k % 4], so that a warp reading entries k..k+3 of
// its 32 particles with one 16-byte load per lane touches 512 consecutive
// bytes.  The list array holds ceil(N / 32) * 32 * cap entries.
__host__ __device__ __forceinline__ int64_t nbr_slot(int64_t i, int k, int cap) {
  return ((((i >> 5) * (int64_t)(cap >> 2) + (k >> 2)) << 5) + (i & 31)) * 4 + (k & 3);
}

// Owner bits of a particle id (bit k for axis k): the top three bits of a
// multiply / xor-shift mix of the id as a 32-bit unsigned integer.  Along an
// axis where a pair's two cells coincide, the bit of the pair's lower id
// picks which of the two blocks holding that coordinate owns the pair: the
// one where the cell is the lower (0) or the upper (1) cell of the block.
__device__ __forceinline__ unsigned owner_bits(int32_t id) {
  uint32_t x = (uint32_t)id;
  x *= 2654435761u;
  x ^= x >> 15;
  x *= 2246822519u;
  x ^= x >> 13;
  x *= 3266489917u;
  x ^= x >> 16;
  return x >> 29;
}

// ---------------------------------------------------------------------------
// Pair distance from r^2.  float64: 1/r from the float32 reciprocal square
// root refined by one Newton step for y = 1/sqrt(x), y <- y (3 - x y^2) / 2
// (quadratic convergence: from the float32 estimate's ~2.4e-7 to ~1e-13
// relative), then r = x y; a handful of float64 operations instead of a
// correctly rounded square root.  r^2 below 1e-30 (coincident particles)
// takes the library square root.  float: r^2 times the hardware reciprocal
// square root (0 for coincident particles).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double pair_rinv(double r2) {
  const double y = (double)rsqrtf((float)r2);
  return y * (1.5 - 0.5 * r2 * y * y);
}
__device__ __forceinline__ double pair_r(double r2) { return r2 > 1e-30 ? r2 * pair_rinv(r2) : sqrt(r2); }
__device__ __forceinline__ float pair_r(float r2) { return r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f; }

// ---------------------------------------------------------------------------
// Smoothing kernels of Section 2.1.1 as functions of x = r/h in [0, 1).
// W: cubic spline of Eq. (sdpd-cubic-w) (cW = 8/(pi h^3)) or Lucy's kernel
// (cW = 105/(16 pi h^3)).  F with grad W = -F(r) r: cubic cF = 48/(pi h^5),
// outer branch (h/r)(1-x)^2; Lucy cF = 315/(4 pi h^5), F = cF (1-x)^2.
// ---------------------------------------------------------------------------
template <int KIND, class R>
__device__ __forceinline__ R kernel_W(R x, R cW) {
  R y = R(1) - x;
  if (KIND == SDPD_KERNEL_LUCY) return cW * (R(1) + R(3) * x) * (y * y * y);
  if (x <= R(0.5)) return cW * (R(1) - R(6) * x * x + R(6) * x * x * x);
  return R(2) * cW * (y * y * y);
}

template <int KIND, class R>
__device__ __forceinline__ R kernel_F(R x, R cF) {
  R y = R(1) - x;
  if (KIND == SDPD_KERNEL_LUCY) return cF * (y * y);
  if (x <= R(0.5)) return cF * (R(2) - R(3) * x);
  return cF * (y * y) / x;
}

// ---------------------------------------------------------------------------
// Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// ten rounds of (multiply words 0 and 2 by the round constants; swap the
// halves, xoring the high halves with words 1, 3 and the key), the key
// advanced by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                              uint64_t k0, uint64_t k1, uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    uint64_t y0 = hi1 ^ c1 ^ k0, y2 = hi0 ^ c3 ^ k1;
    c0 = y0; c1 = lo1; c2 = y2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Random numbers of one pair at one sweep: G ~ N(0, I3) and U ~ U(0,1).
// Key (seed, 0), counter (sweep, id_min, id_max, 0).  Words 0 and 1 give G0,
// G1 by Box-Muller on two uniforms; word 2 gives G2 by Box-Muller on its two
// 32-bit halves; word 3 gives U.  Uniforms are (x + 1/2) 2^-b for the top
// b = 53 bits of a word (32 for the halves of word 2).  The float32 path
// rounds the same uniforms to float32 (pair_randoms_fast).
__device__ __forceinline__ void pair_randoms(uint64_t seed, uint64_t sweep, uint64_t idi, uint64_t idj,
                                             double G[3], double* U) {
  uint64_t w[4];
  philox4x64_10(sweep, idi, idj, 0ull, seed, 0ull, w);
  const double two53 = 1.0 / 9007199254740992.0, two32 = 1.0 / 4294967296.0;
  double u0 = ((double)(w[0] >> 11) + 0.5) * two53;
  double u1 = ((double)(w[1] >> 11) + 0.5) * two53;
  double R = sqrt(-2.0 * log(u0));
  double s, c;
  sincospi(2.0 * u1, &s, &c);
  G[0] = R * c;
  G[1] = R * s;
  double u2 = ((double)(uint32_t)(w[2] >> 32) + 0.5) * two32;
  double u3 = ((double)(uint32_t)(w[2] & 0xffffffffull) + 0.5) * two32;
  G[2] = sqrt(-2.0 * log(u2)) * cospi(2.0 * u3);
  *U = ((double)(w[3] >> 11) + 0.5) * two53;
}

// ---------------------------------------------------------------------------
// Precision policies.
//   Fp64: positions float64 absolute in [0, L); all arithmetic float64.
//   Mixed: positions 32-bit fixed point (x = u * L / 2^32, so the periodic
//   wrap and the minimum image are integer wrap-around); pair arithmetic in
//   float32 on cell-relative coordinates; eps in float64.
// ---------------------------------------------------------------------------
struct alignas(32) D4 { double x, y, z, w; };
struct alignas(16) F4 { float x, y, z, w; };

struct Fp64 {
  using R = double;   // pair arithmetic, momenta, densities
  using V4 = D4;      // (x, y, z, w) records
  using Q = double;   // stored position component
  static constexpr bool mixed = false;
};
struct Mixed {
  using R = float;
  using V4 = F4;
  using Q = uint32_t;
  static constexpr bool mixed = true;
};

// Packed cell coordinates (10 bits per axis).
__host__ __device__ __forceinline__ uint32_t pack_cell(int cx, int cy, int cz) {
  return (uint32_t)cx | ((uint32_t)cy << 10) | ((uint32_t)cz << 20);
}
__host__ __device__ __forceinline__ void unpack_cell(uint32_t c, int& cx, int& cy, int& cz) {
  cx = (int)(c & 1023u); cy = (int)((c >> 10) & 1023u); cz = (int)(c >> 20);
}

__device__ __forceinline__ D4 ld4(const D4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  return D4{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ F4 ld4(const F4* p) {
  float4 a = __ldg(reinterpret_cast<const float4*>(p));
  return F4{a.x, a.y, a.z, a.w};
}
__device__ __forceinline__ void st4(D4* p, const D4& v) {
  double2* q = reinterpret_cast<double2*>(p);
  q[0] = make_double2(v.x, v.y);
  q[1] = make_double2(v.z, v.w);
}
__device__ __forceinline__ void st4(F4* p, const F4& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.x, v.y, v.z, v.w);
}
__device__ __forceinline__ double cellbits_to_w(uint32_t c, D4*) { return (double)c; }
__device__ __forceinline__ float cellbits_to_w(uint32_t c, F4*) { return __uint_as_float(c); }
__device__ __forceinline__ uint32_t w_to_cellbits(double w) { return (uint32_t)w; }
__device__ __forceinline__ uint32_t w_to_cellbits(float w) { return __float_as_uint(w); }

// Periodic wrap into [0, L) for a coordinate at most one box away.
__device__ __forceinline__ double wrap_coord(double x, double L) {
  if (x >= L) x = __dsub_rn(x, L);
  else if (x < 0.0) x = __dadd_rn(x, L);
  if (x >= L || x < 0.0) {  // further away: reduce with floor
    x = x - L * floor(x / L);
    if (x >= L) x = 0.0;
  }
  return x;
}

// Periodic minimum image of a float64 displacement (compare and subtract).
__device__ __forceinline__ double min_image(double d, double L, double halfL) {
  if (d > halfL) return __dsub_rn(d, L);
  if (d < -halfL) return __dadd_rn(d, L);
  return d;
}
// r^2 with the fused multiply-adds written out (fixed rounding sequence).
__device__ __forceinline__ double r2_of(double dx, double dy, double dz) {
  return __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
}
// Periodic image of a neighbour in the cell at offset o in {-1, 0, +1} from
// cell index ci (of n cells, box side L): +L if the offset wraps below 0, -L
// if it wraps above n - 1, else 0.  Neighbour cells are at most one cell
// away, so the float64 displacement (x_i - x_j) + shift equals the minimum
// image (x_i - x_j) -/+ L whenever the pair can be within h: a wrapped
// difference exceeds L/2 in magnitude (n >= 4), an unwrapped one is below it.
__device__ __forceinline__ double image_shift(int ci, int o, int n, double L) {
  return (o < 0 && ci == 0) ? L : ((o > 0 && ci == n - 1) ? -L : 0.0);
}

__device__ __forceinline__ float r2_of(float dx, float dy, float dz) {
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// ---------------------------------------------------------------------------
// Device state of one handle.
// ---------------------------------------------------------------------------
template <class P>
struct Arrays {
  using R = typename P::R;
  using V4 = typename P::V4;
  using Q = typename P::Q;
  V4* q4;      // sorted: (x, y, z, cell bits); mixed: cell-relative float coordinates
  Q* qx;       // sorted positions (float64 absolute or 32-bit fixed point)
  Q* qy;
  Q* qz;
  R* px;
  R* py;
  R* pz;
  double* eps;
  R* rho;
  int32_t* id;
};

struct Workspace {
  // two copies of the sorted state (A = current, B = sort target); typed
  // views are made per precision from these raw pointers
  void* q4[2];
  void* qx[2];
  void* qy[2];
  void* qz[2];
  void* px[2];
  void* py[2];
  void* pz[2];
  double* eps[2];
  void* rho[2];
  int32_t* id[2];
  void* qp4;            // sorted (x, y, z, pi): positions and p/rho^2 for force passes
  void* qr4;            // sorted (x, y, z, rho) of the latest density pass: the sweep's geometry
  float4* qf4;          // float64 path: float32 copies (x, y, z, 0) of the sorted positions
  uint32_t* nlist;      // neighbour lists, entry k of particle i at nlist[nbr_slot(i, k, nbr_cap)]
  int32_t* nn;          // neighbour count per particle
  uint32_t* cend;       // [9][N]: per particle and row of 3 cells, where its list stands (see k_density)
  // binning and sorting scratch
  int32_t* key;         // cell rank per particle (old order)
  int32_t* slot;        // arrival slot in the cell (old order)
  int32_t* tmp;         // bucketed old indices
  void* qdx;            // drifted positions, old order
  void* qdy;
  void* qdz;
  int32_t* cell_count;  // [ncell] (kept zero between uses)
  int32_t* cell_start;  // [ncell + 1]
  int32_t* tile_sum;    // scan scratch: one entry per 2048 cells
  int32_t* mrank;       // linear cell -> Morton rank
  uint32_t* rcoord;     // Morton rank -> packed cell coordinates
  uint32_t* xmin[3];    // mixed: fixed-point lower edge of each cell, per axis
  // pair schedule of the fluctuation/dissipation sweep (per owner cell)
  uint32_t* sched_hdr;    // npairs | nlevels << 16
  uint16_t* sched_lvl;    // [ncell][kMaxLevels + 1] level offsets
  uint16_t* sched_pair;   // [ncell][kMaxPairs] (local min-id | local max-id << 8)
  uint8_t* level_of;      // [ncell][kMaxPairs] level of each pair in canonical order
  // host <-> device staging in id order (float64)
  double* io_q;
  double* io_p;
  double* io_e;
  // reductions and status
  double* obs_partial;        // [kObsBlocks][8]
  double* obs;                // [8]
  unsigned long long* counters;  // [4]: pairs, accept, reject bound, reject metropolis
  unsigned long long* sweep;     // sweep counter: the random-number step of the next sweep
  int* status;
  uint32_t* blk_hist;            // [8][256]: blocks of each colour by dependency depth, then cursors
  int32_t* blk_order;            // [8][ncell / 8]: each colour's blocks, deepest first
  unsigned* fd_queue;            // [8][3]: next block, finished warps and next entry of
                                 // big_list of each colour launch; zero between launches
  int32_t* big_perm;             // [N]: rank order of the particles of blocks beyond capacity
  int2* big_list;                // [8][ncell / 8]: each colour's blocks beyond capacity (owner
                                 // cell, offset in big_perm)
  uint32_t* big_count;           // [8] entries of big_list, then [8] entries of big_perm in use
  // particles whose neighbour list overflows its row, listed by the density
  // pass into one of two slots: [2][N] entries and [2] counts.  A density
  // pass fills slot *ovf_slot (toggled on the host before each launch) and
  // clears the other one, which no kernel reads any more (the force passes
  // read the slot of the latest density pass).
  int32_t* ovf_list;
  int32_t* ovf_count;
  int* ovf_slot;                 // host: the slot of the latest density pass
  sdpd_pair_rec* pair_recs;   // debug
  unsigned long long* pair_rec_count;
  int64_t pair_rec_cap;
};

constexpr int kObsBlocks = 304;

template <class P>
Arrays<P> view(const Workspace& w, int k) {
  Arrays<P> a;
  a.q4 = (typename P::V4*)w.q4[k];
  a.qx = (typename P::Q*)w.qx[k];
  a.qy = (typename P::Q*)w.qy[k];
  a.qz = (typename P::Q*)w.qz[k];
  a.px = (typename P::R*)w.px[k];
  a.py = (typename P::R*)w.py[k];
  a.pz = (typename P::R*)w.pz[k];
  a.eps = w.eps[k];
  a.rho = (typename P::R*)w.rho[k];
  a.id = w.id[k];
  return a;
}

// ---------------------------------------------------------------------------
// Launchers (host side), one per pipeline stage; P in {Fp64, Mixed}.
// ---------------------------------------------------------------------------
template <class P>
void launch_load(const Consts& c, const Workspace& w, cudaStream_t s);
template <class P>
void launch_sort(const Consts& c, const Workspace& w, int from, cudaStream_t s);
template <class P>
void launch_unload(const Consts& c, const Workspace& w, int cur, cudaStream_t s);
template <class P>
void launch_density(const Consts& c, const Workspace& w, int cur, int update_eos, int32_t* ncount_by_id,
                    cudaStream_t s);
template <class P>
void launch_force(const Consts& c, const Workspace& w, int cur, double half_dt, double dt_drift,
                  double* force_by_id, cudaStream_t s);
template <class P>
void launch_fd_schedule(const Consts& c, const Workspace& w, int cur, cudaStream_t s);
// the sweep's colour launches: P the state's storage policy, A the pair
// arithmetic (A = Mixed on float64 state: float32 pair updates)
template <class P, class A = P>
void fd_prepare();
template <class P, class A = P>
void launch_fd_colours(const Consts& c, const Workspace& w, int cur, double dt, uint64_t seed, int record,
                       cudaStream_t s);
template <class P>
void launch_observables(const Consts& c, const Workspace& w, int cur, cudaStream_t s);
// sweep counter on the device: set to a value, or advanced by one
void launch_set_sweep(const Workspace& w, unsigned long long value, cudaStream_t s);
void launch_advance_sweep(const Workspace& w, cudaStream_t s);

// Reverse-mode passes (float64 storage layout, after a density pass has built
// qp4 = (q, pi) and the neighbour lists).  vs4[i] = (v_i, rbar_i) in storage
// order; qbar, pbar, Sbar, thbar (per-particle (h, c_rho, C_K) terms) in id
// order.  mode: 0 kick pulled back along v, 1 virial, 2 density term only.
void launch_adj_gather(const Consts& c, const Workspace& w, int cur, const double* pbar_id, double scale, D4* vs4,
                       cudaStream_t s);
void launch_adj_pairsum(const Consts& c, const Workspace& w, int cur, int mode, const D4* vs4, double* A,
                        cudaStream_t s);
void launch_adj_mid_step(const Consts& c, const Workspace& w, int cur, const double* A, bool kick1, bool kick2,
                         const double* deps_prev, double* Sbar_cur, double* Sbar_prev, const double* epsbar_n,
                         double* epsbar0, D4* vs4, double* thbar, cudaStream_t s);
// frozen sweeps: record (increments stored, state set to before + increment)
// and replay (increments added); pre = the sorted px, py, pz, eps before
void launch_adj_freeze(const Consts& c, const Workspace& w, int cur, const double* pre, double* dp, double* de,
                       cudaStream_t s);
void launch_adj_increment(const Consts& c, const Workspace& w, int cur, const double* dp, const double* de,
                          cudaStream_t s);
void launch_adj_mid_virial(const Consts& c, const Workspace& w, int cur, const double* A, double wt, D4* vs4,
                           double* val_id, double* gp, double* geps, double* thbar, cudaStream_t s);
void launch_adj_back(const Consts& c, const Workspace& w, int cur, int mode, double wt, const D4* vs4,
                     int accumulate, double* qbar, double* thbar, cudaStream_t s);
void launch_adj_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s);
size_t adj_sum_partial_doubles();
// histogram of eps * scale (sdpd_stats.cu): nbins bins over [lo, hi), then
// the counts below lo and at or above hi; adds into counts[nbins + 2]
void launch_energy_hist(const Consts& c, const Workspace& w, int cur, double lo, double hi, int nbins,
                        double scale, unsigned long long* counts, cudaStream_t s);
void launch_adj_sum(const double* x, int64_t n, int ncols, double* partial, double* out, cudaStream_t s);

}  // namespace sdpd
