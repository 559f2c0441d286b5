// sdpd_api.cu -- the C ABI of include/sdpd.h: parameter checks, workspace
// layout, cell tables, the time-step driver and the float64 observables.
#include <float.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <type_traits>
#include <vector>

#include "sdpd_internal.cuh"

using namespace sdpd;

struct sdpd_handle {
  Consts c;
  sdpd_params prm;
  double K;
  cudaStream_t stream;
  size_t ws_bytes;
  char* ws;
  Workspace w;
  int cur;
  bool has_state;
  int64_t fd_step, vv_step;
  int64_t launches;
  // the sweep schedule on the device matches the current positions (it
  // depends on them only; it is reused by the sweeps of FD-only runs)
  bool sched_valid = false;
  std::vector<int32_t> mrank_h;
  std::vector<uint32_t> rcoord_h;
  std::vector<uint32_t> xmin_h[3];
  int64_t pair_rec_cap;
  int device;  // device of the bound workspace; selected on entry to every call
  int ovf_slot = 0;  // slot of the neighbour-list overflow list of the latest density pass
  // stage timing: event pairs recorded on the stream, reduced at sync points
  bool timing;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double stage_ms[SDPD_NSTAGES];
  int64_t stage_launches[SDPD_NSTAGES];
  // the trajectory last recorded by sdpd_vv_record (for sdpd_vv_adjoint)
  struct {
    const void* tape = nullptr;
    size_t bytes = 0;
    int64_t nsteps = 0, every = 1;
    double dt = 0.0;
  } rec;
};

namespace {

constexpr size_t kAlign = 256;

struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + kAlign - 1) / kAlign * kAlign;
    return o;
  }
};

// Interleave the bits of (x, y, z), x lowest: the Morton code of a cell.
uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  uint64_t code = 0;
  for (int b = 0; b < 21; ++b) {
    code |= (uint64_t)((x >> b) & 1u) << (3 * b);
    code |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
    code |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
  }
  return code;
}

int map_status(int bits) {
  if (bits & kStNaN) return SDPD_ERR_NAN;
  if (bits & kStNegative) return SDPD_ERR_NEGATIVE_ENERGY;
  if (bits & (kStCapacity | kStNbrCap)) return SDPD_ERR_CAPACITY;
  if (bits & kStBadEnergy) return SDPD_ERR_NONPOSITIVE_ENERGY;
  return SDPD_OK;
}

// Observables: per-block float64 partial sums, then one block in fixed order.
// slots: 0 sum eps, 1 kinetic energy, 2..4 momentum, 5 sum T, 6 min eps,
// 7 non-finite flag.
template <class P>
__global__ void k_obs_partial(Consts c, Arrays<P> a, double* partial) {
  double s[6] = {0, 0, 0, 0, 0, 0};
  double emin = INFINITY, bad = 0.0;
  const double inv2m = 0.5 / c.m, invCK = 1.0 / c.C_K;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.N; i += (int64_t)gridDim.x * blockDim.x) {
    const double e = a.eps[i];
    const double px = a.px[i], py = a.py[i], pz = a.pz[i];
    s[0] += e;
    s[1] += (px * px + py * py + pz * pz) * inv2m;
    s[2] += px; s[3] += py; s[4] += pz;
    s[5] += e * invCK;
    emin = fmin(emin, e);
    if (!isfinite(e) || !isfinite(px) || !isfinite(py) || !isfinite(pz)) bad = 1.0;
  }
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double v[8] = {s[0], s[1], s[2], s[3], s[4], s[5], emin, bad};
  for (int k = 0; k < 8; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) {
      double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = (k == 6) ? fmin(x, y) : (k == 7 ? fmax(x, y) : x + y);
    }
    if (lane == 0) red[k][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < 8; ++k) {
      double x = lane < nw ? red[k][lane] : (k == 6 ? INFINITY : 0.0);
      for (int o = 16; o > 0; o >>= 1) {
        double y = __shfl_xor_sync(0xffffffffu, x, o);
        x = (k == 6) ? fmin(x, y) : (k == 7 ? fmax(x, y) : x + y);
      }
      if (lane == 0) partial[blockIdx.x * 8 + k] = x;
    }
  }
}

__global__ void k_obs_final(const double* partial, int nb, double* out, int* status) {
  const int lane = threadIdx.x;
  for (int k = 0; k < 8; ++k) {
    double x = (k == 6) ? INFINITY : 0.0;
    for (int b = lane; b < nb; b += 32) {
      const double y = partial[b * 8 + k];
      x = (k == 6) ? fmin(x, y) : (k == 7 ? fmax(x, y) : x + y);
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = (k == 6) ? fmin(x, y) : (k == 7 ? fmax(x, y) : x + y);
    }
    if (lane == 0) out[k] = x;
  }
  if (lane == 0 && out[7] != 0.0) atomicOr(status, kStNaN);
}

template <class P>
size_t layout(sdpd_handle* s, Workspace* w, char* base) {
  const Consts& c = s->c;
  using R = typename P::R;
  using Q = typename P::Q;
  using V4 = typename P::V4;
  const size_t N = (size_t)(c.N > 0 ? c.N : 1);
  const size_t nc = (size_t)c.ncell;
  Layout L;
  auto at = [&](size_t bytes) -> void* { return base ? base + L.take(bytes) : (L.take(bytes), nullptr); };
  for (int k = 0; k < 2; ++k) {
    w->q4[k] = at(N * sizeof(V4));
    w->qx[k] = at(N * sizeof(Q));
    w->qy[k] = at(N * sizeof(Q));
    w->qz[k] = at(N * sizeof(Q));
    w->px[k] = at(N * sizeof(R));
    w->py[k] = at(N * sizeof(R));
    w->pz[k] = at(N * sizeof(R));
    w->eps[k] = (double*)at(N * sizeof(double));
    w->rho[k] = at(N * sizeof(R));
    w->id[k] = (int32_t*)at(N * sizeof(int32_t));
  }
  w->qp4 = at(N * sizeof(V4));
  w->qr4 = at(N * sizeof(V4));
  w->qf4 = P::mixed ? nullptr : (float4*)at(N * sizeof(float4));
  w->nlist = (uint32_t*)at((N + 31) / 32 * 32 * (size_t)c.nbr_cap * 4);
  w->nn = (int32_t*)at(N * 4);
  w->cend = (uint32_t*)at(9 * N * 4);
  w->key = (int32_t*)at(N * 4);
  w->slot = (int32_t*)at(N * 4);
  w->tmp = (int32_t*)at(2 * N * 4);
  w->qdx = at(N * sizeof(Q));
  w->qdy = at(N * sizeof(Q));
  w->qdz = at(N * sizeof(Q));
  w->cell_count = (int32_t*)at(nc * 4);
  w->cell_start = (int32_t*)at((nc + 1) * 4);
  w->tile_sum = (int32_t*)at((nc / 2048 + 2) * 4);
  w->mrank = (int32_t*)at(nc * 4);
  w->rcoord = (uint32_t*)at(nc * 4);
  for (int d = 0; d < 3; ++d) w->xmin[d] = (uint32_t*)at((size_t)c.nc[d] * 4);
  w->sched_hdr = (uint32_t*)at(nc * 4);
  w->sched_lvl = (uint16_t*)at(nc * (kMaxLevels + 1) * 2);
  w->sched_pair = (uint16_t*)at(2 * nc * kMaxPairs * 2);
  w->level_of = (uint8_t*)at(nc * kMaxPairs);
  w->io_q = (double*)at(3 * N * 8);
  w->io_p = (double*)at(3 * N * 8);
  w->io_e = (double*)at(N * 8);
  w->obs_partial = (double*)at(kObsBlocks * 8 * 8);
  w->obs = (double*)at(16 * 8);
  w->counters = (unsigned long long*)at(4 * 8);
  w->sweep = (unsigned long long*)at(8);
  w->status = (int*)at(8);
  w->fd_queue = (unsigned*)at(32 * 4);
  w->big_perm = (int32_t*)at(N * 4);
  w->big_list = (int2*)at(nc * 8);
  w->big_count = (uint32_t*)at(16 * 4);
  w->ovf_list = (int32_t*)at(2 * N * 4);
  w->ovf_count = (int32_t*)at(2 * 4);
  w->ovf_slot = &s->ovf_slot;
  w->blk_hist = (uint32_t*)at(8 * 256 * 4);
  w->blk_order = (int32_t*)at(nc * 4);
  w->pair_rec_count = (unsigned long long*)at(8);
  w->pair_rec_cap = s->pair_rec_cap;
  w->pair_recs = s->pair_rec_cap > 0 ? (sdpd_pair_rec*)at((size_t)s->pair_rec_cap * sizeof(sdpd_pair_rec)) : nullptr;
  return L.off;
}

size_t layout_any(sdpd_handle* s, Workspace* w, char* base) {
  return s->prm.precision == SDPD_MIXED ? layout<Mixed>(s, w, base) : layout<Fp64>(s, w, base);
}

int cuda_ok(cudaError_t e) { return e == cudaSuccess ? SDPD_OK : SDPD_ERR_CUDA; }

// Make the workspace's device current for this runtime on the calling thread.
int use_device(sdpd_handle* s) {
  if (s->device < 0) return SDPD_OK;
  int cur = -1;
  if (cudaGetDevice(&cur) == cudaSuccess && cur == s->device) return SDPD_OK;
  return cuda_ok(cudaSetDevice(s->device));
}

int launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SDPD_OK : SDPD_ERR_CUDA;
}

template <class P>
void do_load(sdpd_handle* s) {
  launch_load<P>(s->c, s->w, s->stream);
  launch_sort<P>(s->c, s->w, 0, s->stream);
  s->cur = 1;
  launch_density<P>(s->c, s->w, s->cur, 0, nullptr, s->stream);
  s->launches += 7;
  s->sched_valid = false;
}

cudaEvent_t take_event(sdpd_handle* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Reduce the recorded event pairs (the stream must be synchronised).
void drain_events(sdpd_handle* s) {
  for (auto& it : s->ev_pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, it.second.first, it.second.second) == cudaSuccess) s->stage_ms[it.first] += ms;
    s->ev_pool.push_back(it.second.first);
    s->ev_pool.push_back(it.second.second);
  }
  s->ev_pending.clear();
}

// Reduce the event pairs that the device has already passed, oldest first,
// without waiting for the rest: the stage timers never block the host.
void drain_completed_events(sdpd_handle* s) {
  size_t k = 0;
  for (; k < s->ev_pending.size(); ++k) {
    auto& it = s->ev_pending[k];
    if (cudaEventQuery(it.second.second) != cudaSuccess) break;  // not reached yet (cudaErrorNotReady)
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, it.second.first, it.second.second) == cudaSuccess) s->stage_ms[it.first] += ms;
    s->ev_pool.push_back(it.second.first);
    s->ev_pool.push_back(it.second.second);
  }
  s->ev_pending.erase(s->ev_pending.begin(), s->ev_pending.begin() + (ptrdiff_t)k);
}

// Brackets one stage with events when timing is on.  The pending pairs are
// reduced when the device has passed them (checked without blocking every
// 256 pairs) or at the next synchronising call; the event pool grows
// meanwhile instead of waiting.
struct StageTimer {
  sdpd_handle* s;
  int stage;
  int launches;
  cudaEvent_t a = nullptr;
  StageTimer(sdpd_handle* s_, int st, int nl) : s(s_), stage(st), launches(nl) {
    if (s->timing) {
      a = take_event(s);
      cudaEventRecord(a, s->stream);
    }
  }
  ~StageTimer() {
    if (s->timing) {
      cudaEvent_t b = take_event(s);
      cudaEventRecord(b, s->stream);
      s->ev_pending.push_back({stage, {a, b}});
      s->stage_launches[stage] += launches;
      if (s->ev_pending.size() % 256 == 0) drain_completed_events(s);
    }
  }
};

// One Velocity Verlet step, Eq. (sdpd-verlet), at fixed entropies.
template <class P>
void vv_step(sdpd_handle* s, double dt) {
  const Consts& c = s->c;
  {  // p^{n+1/2} = p^n + F^n dt/2, q^{n+1} = q^n + p^{n+1/2} dt/m
    StageTimer t(s, 0, 2);
    launch_force<P>(c, s->w, s->cur, 0.5 * dt, dt, nullptr, s->stream);
  }
  {
    StageTimer t(s, 1, 5);
    launch_sort<P>(c, s->w, s->cur, s->stream);
  }
  s->cur = 1 - s->cur;
  {  // rho^{n+1}, eps^{n+1} = E(S, rho^{n+1})
    StageTimer t(s, 2, 1);
    launch_density<P>(c, s->w, s->cur, 1, nullptr, s->stream);
  }
  {  // p^{n+1} = p^{n+1/2} + F^{n+1} dt/2
    StageTimer t(s, 3, 2);
    launch_force<P>(c, s->w, s->cur, 0.5 * dt, 0.0, nullptr, s->stream);
  }
  s->launches += 10;  // force + overflow, 5 sort, density, force + overflow
  s->vv_step++;
  s->sched_valid = false;
}

// MTS: one sweep after every theta-th Verlet step since sdpd_set_state
// (after every step in FD-only runs).
bool sweep_due(const sdpd_handle* s) {
  const int theta = s->prm.theta < 1 ? 1 : s->prm.theta;
  return s->prm.scheme != SDPD_SCHEME_NONE && (s->prm.fd_only || s->vv_step % theta == 0);
}

// Whether the sweep's pair arithmetic is float32 (the mixed path, or a
// float64 state swept in float32).
bool sweep_float(const sdpd_handle* s) { return s->prm.precision == SDPD_MIXED || s->prm.sweep_f32 != 0; }

// One fluctuation/dissipation sweep with step dt_fd.
template <class P>
void fd_sweep_step(sdpd_handle* s, double dt_fd, uint64_t seed) {
  const Consts& c = s->c;
  const int rec = s->w.pair_recs != nullptr;
  if (rec) cudaMemsetAsync(s->w.pair_rec_count, 0, 8, s->stream);
  if (!s->sched_valid) {  // positions unchanged since the last sweep: reuse it
    StageTimer t(s, 4, 5);
    launch_fd_schedule<P>(c, s->w, s->cur, s->stream);
    s->launches += 5;
    s->sched_valid = true;
  }
  {
    StageTimer t(s, 5, 8);
    if constexpr (std::is_same<P, Fp64>::value) {
      if (s->prm.sweep_f32) launch_fd_colours<Fp64, Mixed>(c, s->w, s->cur, dt_fd, seed, rec, s->stream);
      else launch_fd_colours<Fp64, Fp64>(c, s->w, s->cur, dt_fd, seed, rec, s->stream);
    } else {
      launch_fd_colours<P, P>(c, s->w, s->cur, dt_fd, seed, rec, s->stream);
    }
  }
  launch_advance_sweep(s->w, s->stream);
  s->launches += 9;
  s->fd_step++;
}

template <class P>
void do_steps(sdpd_handle* s, double dt, int64_t nsteps, uint64_t seed) {
  const int theta = s->prm.theta < 1 ? 1 : s->prm.theta;
  for (int64_t n = 0; n < nsteps; ++n) {
    if (!s->prm.fd_only) vv_step<P>(s, dt);
    if (sweep_due(s)) fd_sweep_step<P>(s, s->prm.fd_only ? dt : theta * dt, seed);
  }
}

template <class P>
void do_observables(sdpd_handle* s) {
  launch_observables<P>(s->c, s->w, s->cur, s->stream);
  s->launches += 2;
}

}  // namespace

namespace sdpd {
template <class P>
void launch_observables(const Consts& c, const Workspace& w, int cur, cudaStream_t s) {
  k_obs_partial<P><<<kObsBlocks, 256, 0, s>>>(c, view<P>(w, cur), w.obs_partial);
  k_obs_final<<<1, 32, 0, s>>>(w.obs_partial, kObsBlocks, w.obs, w.status);
}
template void launch_observables<Fp64>(const Consts&, const Workspace&, int, cudaStream_t);
template void launch_observables<Mixed>(const Consts&, const Workspace&, int, cudaStream_t);
}  // namespace sdpd

extern "C" {

const char* sdpd_strerror(int st) {
  switch (st) {
    case SDPD_OK: return "ok";
    case SDPD_ERR_INVALID_ARG: return "invalid argument";
    case SDPD_ERR_BOX_TOO_SMALL: return "box too small: need an even number >= 4 of cells of side >= h per axis";
    case SDPD_ERR_NONPOSITIVE_ENERGY: return "internal energy <= 0 or not finite in the given state";
    case SDPD_ERR_NEGATIVE_ENERGY: return "SSA produced a non-positive internal energy";
    case SDPD_ERR_NAN: return "non-finite momentum or energy";
    case SDPD_ERR_CUDA: return "CUDA runtime error";
    case SDPD_ERR_TIMEOUT: return "bounded device wait ran out";
    case SDPD_ERR_NO_WORKSPACE: return "no or too small workspace bound";
    case SDPD_ERR_CAPACITY: return "a 2x2x2 cell block exceeded its particle or pair capacity";
    case SDPD_ERR_NO_STATE: return "no state loaded";
    case SDPD_ERR_HOST_MEMORY: return "host memory allocation failed";
    default: return "unknown status";
  }
}

int sdpd_create(int64_t N, const double box[3], double m, double h, const sdpd_params* prm, double K,
                void* stream, sdpd_t** out) {
  if (!out) return SDPD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!box || !prm) return SDPD_ERR_INVALID_ARG;
  if (N < 0 || N >= (int64_t)INT32_MAX) return SDPD_ERR_INVALID_ARG;
  if (!(m > 0) || !isfinite(m) || !(h > 0) || !isfinite(h)) return SDPD_ERR_INVALID_ARG;
  if (!(K > 4.0 / 3.0) || !isfinite(K)) return SDPD_ERR_INVALID_ARG;
  if (!(prm->kB > 0) || !isfinite(prm->kB)) return SDPD_ERR_INVALID_ARG;
  if (!(prm->eta > 0) || !isfinite(prm->eta)) return SDPD_ERR_INVALID_ARG;
  if (!(prm->zeta >= 0) || !(prm->zeta < 5.0 * prm->eta / 3.0)) return SDPD_ERR_INVALID_ARG;
  if (prm->kernel != SDPD_KERNEL_CUBIC && prm->kernel != SDPD_KERNEL_LUCY) return SDPD_ERR_INVALID_ARG;
  if (prm->scheme < SDPD_SCHEME_SSA || prm->scheme > SDPD_SCHEME_NONE) return SDPD_ERR_INVALID_ARG;
  if (prm->precision != SDPD_FP64 && prm->precision != SDPD_MIXED) return SDPD_ERR_INVALID_ARG;
  if (prm->theta < 1 || prm->theta > 1000000) return SDPD_ERR_INVALID_ARG;
  if (prm->fd_only && prm->scheme == SDPD_SCHEME_NONE) return SDPD_ERR_INVALID_ARG;
  sdpd_handle* s = new (std::nothrow) sdpd_handle();
  if (!s) return SDPD_ERR_INVALID_ARG;
  Consts& c = s->c;
  c.N = N;
  int64_t ncell = 1;
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0) || !isfinite(box[d])) { delete s; return SDPD_ERR_INVALID_ARG; }
    int64_t n;
    if (prm->nc[d] != 0) {  // a chosen grid: even, >= 4, cells of side >= h
      n = prm->nc[d];
      if (n < 4 || n % 2 != 0 || n > 1024) { delete s; return SDPD_ERR_INVALID_ARG; }
      if (box[d] / (double)n < h) { delete s; return SDPD_ERR_BOX_TOO_SMALL; }
    } else {
      double ratio = floor(box[d] / h);
      n = ratio > 1024.0 ? 1024 : (int64_t)ratio;
      n -= n % 2;
      if (n < 4) { delete s; return SDPD_ERR_BOX_TOO_SMALL; }
    }
    c.nc[d] = (int)n;
    c.L[d] = box[d];
    c.halfL[d] = 0.5 * box[d];
    c.cs[d] = box[d] / (double)n;
    c.scale[d] = box[d] / 4294967296.0;
    c.inv_scale[d] = 4294967296.0 / box[d];
    ncell *= n;
  }
  c.ncell = (int)ncell;
  c.h = h;
  c.h2 = h * h;
  c.m = m;
  c.kB = prm->kB;
  c.C_K = 1.5 * (K - 1.0) * prm->kB;
  c.c_rho = prm->c_rho < 0 ? 0.5 * (K - 1.0) : prm->c_rho;
  c.kpar_m2 = (10.0 / 3.0 * prm->eta + 4.0 * prm->zeta) * m * m;
  c.kperp_m2 = (5.0 / 3.0 * prm->eta - prm->zeta) * m * m;
  const double h3 = h * h * h, h5 = h3 * h * h;
  if (prm->kernel == SDPD_KERNEL_LUCY) {
    c.cW = 105.0 / (16.0 * M_PI * h3);
    c.cF = 315.0 / (4.0 * M_PI * h5);
  } else {
    c.cW = 8.0 / (M_PI * h3);
    c.cF = 48.0 / (M_PI * h5);
  }
  c.W0 = c.cW;
  c.nbr_cap = 160;
  {
    // Float32 pre-test of r^2 < h^2 (float64 path).  With u = 2^-24, each
    // float32 coordinate, the float32 difference and the float32 minimum
    // image are within D = 8 u L_max of the float64 displacement's image
    // (three conversions and three roundings of size <= u L, with margin; an
    // image chosen differently only where both images are within D of L/2),
    // so |d_f| <= |d| + 3D per axis and the float32 r_f^2 <= (1 + 8u)
    // (r + 3 sqrt(3) D)^2.  Hence r < h implies r_f^2 < h2_filter below.
    const double u = 0x1.0p-24;
    const double Lmax = std::max(c.L[0], std::max(c.L[1], c.L[2]));
    const double D = 8.0 * u * Lmax;
    const double rf = h + 3.0 * sqrt(3.0) * D;
    c.h2_filter = nextafterf((float)((1.0 + 8.0 * u) * rf * rf), INFINITY);
    for (int d = 0; d < 3; ++d) {
      c.Lf[d] = (float)c.L[d];
      c.halfLf[d] = 0.5f * c.Lf[d];
    }
  }
  c.kernel = prm->kernel;
  c.fd_variant = fd_default_variant(prm->precision == SDPD_MIXED || prm->sweep_f32 != 0);
  c.pair_threads = 128;
  c.scheme = prm->scheme;
  s->prm = *prm;
  s->K = K;
  s->stream = (cudaStream_t)stream;
  s->ws = nullptr;
  s->cur = 0;
  s->has_state = false;
  s->fd_step = s->vv_step = 0;
  s->launches = 0;
  s->pair_rec_cap = prm->debug ? std::max<int64_t>(1, N) * 64 : 0;
  s->timing = false;
  s->device = -1;
  for (int k = 0; k < SDPD_NSTAGES; ++k) { s->stage_ms[k] = 0.0; s->stage_launches[k] = 0; }
  // Morton order of the cells: rank of every cell, and the cell of every rank
  std::vector<std::pair<uint64_t, int64_t>> codes;
  try {
    s->mrank_h.resize((size_t)ncell);
    s->rcoord_h.resize((size_t)ncell);
    codes.resize((size_t)ncell);
    for (int d = 0; d < 3; ++d) s->xmin_h[d].resize((size_t)c.nc[d]);
  } catch (const std::bad_alloc&) {
    delete s;
    return SDPD_ERR_HOST_MEMORY;
  }
  for (int z = 0; z < c.nc[2]; ++z)
    for (int y = 0; y < c.nc[1]; ++y)
      for (int x = 0; x < c.nc[0]; ++x) {
        int64_t lin = x + (int64_t)c.nc[0] * (y + (int64_t)c.nc[1] * z);
        codes[(size_t)lin] = {morton3(x, y, z), lin};
      }
  std::sort(codes.begin(), codes.end());
  for (int64_t r = 0; r < ncell; ++r) {
    int64_t lin = codes[(size_t)r].second;
    int x = (int)(lin % c.nc[0]), y = (int)((lin / c.nc[0]) % c.nc[1]), z = (int)(lin / ((int64_t)c.nc[0] * c.nc[1]));
    s->mrank_h[(size_t)lin] = (int32_t)r;
    s->rcoord_h[(size_t)r] = pack_cell(x, y, z);
  }
  // fixed-point lower edge of each cell: ceil(c 2^32 / n_c)
  for (int d = 0; d < 3; ++d) {
    for (int k = 0; k < c.nc[d]; ++k) {
      uint64_t num = ((uint64_t)k << 32) + (uint64_t)c.nc[d] - 1;
      s->xmin_h[d][(size_t)k] = (uint32_t)(num / (uint64_t)c.nc[d]);
    }
  }
  s->ws_bytes = layout_any(s, &s->w, nullptr);
  *out = s;
  return SDPD_OK;
}

size_t sdpd_workspace_bytes(const sdpd_t* s) { return s ? s->ws_bytes : 0; }

int sdpd_bind_workspace(sdpd_t* s, void* ptr, size_t bytes) {
  if (!s) return SDPD_ERR_INVALID_ARG;
  if (!ptr || bytes < s->ws_bytes || ((uintptr_t)ptr % kAlign) != 0) return SDPD_ERR_NO_WORKSPACE;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return SDPD_ERR_NO_WORKSPACE;
  }
  s->device = attr.device;
  if (use_device(s) != SDPD_OK) return SDPD_ERR_CUDA;
  s->ws = (char*)ptr;
  s->sched_valid = false;
  layout_any(s, &s->w, s->ws);
  const Consts& c = s->c;
  cudaStream_t st = s->stream;
  int e = SDPD_OK;
  e |= cuda_ok(cudaMemcpyAsync(s->w.mrank, s->mrank_h.data(), (size_t)c.ncell * 4, cudaMemcpyHostToDevice, st));
  e |= cuda_ok(cudaMemcpyAsync(s->w.rcoord, s->rcoord_h.data(), (size_t)c.ncell * 4, cudaMemcpyHostToDevice, st));
  for (int d = 0; d < 3; ++d)
    e |= cuda_ok(cudaMemcpyAsync(s->w.xmin[d], s->xmin_h[d].data(), (size_t)c.nc[d] * 4, cudaMemcpyHostToDevice, st));
  e |= cuda_ok(cudaMemsetAsync(s->w.cell_count, 0, (size_t)c.ncell * 4, st));
  e |= cuda_ok(cudaMemsetAsync(s->w.counters, 0, 4 * 8, st));
  e |= cuda_ok(cudaMemsetAsync(s->w.status, 0, 8, st));
  e |= cuda_ok(cudaMemsetAsync(s->w.sched_hdr, 0, (size_t)c.ncell * 4, st));
  e |= cuda_ok(cudaMemsetAsync(s->w.fd_queue, 0, 32 * 4, st));
  e |= cuda_ok(cudaMemsetAsync(s->w.ovf_count, 0, 2 * 4, st));
  e |= cuda_ok(cudaStreamSynchronize(st));
  // launch sizes of the sweep's colour kernels, queried here rather than
  // inside a later stream capture
  if (s->prm.precision == SDPD_MIXED) fd_prepare<Mixed, Mixed>();
  else if (s->prm.sweep_f32) fd_prepare<Fp64, Mixed>();
  else fd_prepare<Fp64, Fp64>();
  e |= launch_status();
  s->has_state = false;
  return e ? SDPD_ERR_CUDA : SDPD_OK;
}

int sdpd_set_state(sdpd_t* s, const double* q, const double* p, const double* eps, int on_device) {
  if (!s) return SDPD_ERR_INVALID_ARG;
  if (!s->ws) return SDPD_ERR_NO_WORKSPACE;
  if (use_device(s) != SDPD_OK) return SDPD_ERR_CUDA;
  const int64_t N = s->c.N;
  if (N > 0 && (!q || !p || !eps)) return SDPD_ERR_INVALID_ARG;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  int e = SDPD_OK;
  cudaStream_t st = s->stream;
  // the copies go to staging buffers only, so they can start before the
  // host check (which overlaps them for pinned memory): a rejected state
  // launches no kernel and leaves the loaded state as it was
  if (N > 0) {
    e |= cuda_ok(cudaMemcpyAsync(s->w.io_q, q, (size_t)N * 3 * 8, kind, st));
    e |= cuda_ok(cudaMemcpyAsync(s->w.io_p, p, (size_t)N * 3 * 8, kind, st));
    e |= cuda_ok(cudaMemcpyAsync(s->w.io_e, eps, (size_t)N * 8, kind, st));
  }
  if (!on_device) {
    int bad = 0;  // eps_i > 0 and finite (NaN fails both comparisons), without branches
    for (int64_t i = 0; i < N; ++i) bad |= (int)!((eps[i] > 0.0) & (eps[i] <= DBL_MAX));
    if (bad) {
      if (cudaStreamSynchronize(st) != cudaSuccess) return SDPD_ERR_CUDA;  // the copies read the caller's memory
      return SDPD_ERR_NONPOSITIVE_ENERGY;
    }
  }
  e |= cuda_ok(cudaMemsetAsync(s->w.counters, 0, 4 * 8, st));
  e |= cuda_ok(cudaMemsetAsync(s->w.status, 0, 8, st));
  e |= cuda_ok(cudaMemsetAsync(s->w.fd_queue, 0, 32 * 4, st));
  if (e) return SDPD_ERR_CUDA;
  if (s->prm.precision == SDPD_MIXED) do_load<Mixed>(s);
  else do_load<Fp64>(s);
  launch_set_sweep(s->w, 0ull, st);
  s->launches += 1;
  if (!on_device && N > 0) {
    // host buffers may be reused by the caller as soon as we return
    if (cudaStreamSynchronize(st) != cudaSuccess) return SDPD_ERR_CUDA;
  }
  s->fd_step = 0;
  s->vv_step = 0;
  s->has_state = true;
  return launch_status();
}

int sdpd_get_state(sdpd_t* s, double* q, double* p, double* eps, int on_device) {
  if (!s) return SDPD_ERR_INVALID_ARG;
  if (!s->ws) return SDPD_ERR_NO_WORKSPACE;
  if (use_device(s) != SDPD_OK) return SDPD_ERR_CUDA;
  if (!s->has_state) return SDPD_ERR_NO_STATE;
  const int64_t N = s->c.N;
  cudaStream_t st = s->stream;
  if (s->prm.precision == SDPD_MIXED) launch_unload<Mixed>(s->c, s->w, s->cur, st);
  else launch_unload<Fp64>(s->c, s->w, s->cur, st);
  s->launches += 1;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  int e = SDPD_OK;
  if (N > 0) {
    if (q) e |= cuda_ok(cudaMemcpyAsync(q, s->w.io_q, (size_t)N * 3 * 8, kind, st));
    if (p) e |= cuda_ok(cudaMemcpyAsync(p, s->w.io_p, (size_t)N * 3 * 8, kind, st));
    if (eps) e |= cuda_ok(cudaMemcpyAsync(eps, s->w.io_e, (size_t)N * 8, kind, st));
  }
  if (e) return SDPD_ERR_CUDA;
  return sdpd_sync(s);
}

int sdpd_step(sdpd_t* s, double dt, int64_t nsteps, uint64_t seed) {
  if (!s) return SDPD_ERR_INVALID_ARG;
  if (!(dt > 0) || !isfinite(dt) || nsteps < 0) return SDPD_ERR_INVALID_ARG;
  if (!s->ws) return SDPD_ERR_NO_WORKSPACE;
  if (use_device(s) != SDPD_OK) return SDPD_ERR_CUDA;
  if (!s->has_state) return SDPD_ERR_NO_STATE;
  if (s->prm.precision == SDPD_MIXED) do_steps<Mixed>(s, dt, nsteps, seed);
  else do_steps<Fp64>(s, dt, nsteps, seed);
  return launch_status();
}

int sdpd_sync(sdpd_t* s) {
  if (!s) return SDPD_ERR_INVALID_ARG;
  if (!s->ws) return SDPD_ERR_NO_WORKSPACE;
  if (use_device(s) != SDPD_OK) return SDPD_ERR_CUDA;
  int bits = 0;
  if (cudaMemcpyAsync(&bits, s->w.status, sizeof(int), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return SDPD_ERR_CUDA;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return SDPD_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return SDPD_ERR_CUDA;
  return map_status(bits);
}

int sdpd_observables(sdpd_t* s, sdpd_obs* out) {
  if (!s || !out) return SDPD_ERR_INVALID_ARG;
  if (!s->ws) return SDPD_ERR_NO_WORKSPACE;
  if (use_device(s) != SDPD_OK) return SDPD_ERR_CUDA;
  if (!s->has_state) return SDPD_ERR_NO_STATE;
  memset(out, 0, sizeof(*out));
  if (s->prm.precision == SDPD_MIXED) do_observables<Mixed>(s);
  else do_observables<Fp64>(s);
  double o[8];
  unsigned long long cnt[4];
  if (cudaMemcpyAsync(o, s->w.obs, sizeof(o), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(cnt, s->w.counters, sizeof(cnt), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return SDPD_ERR_CUDA;
  int st = sdpd_sync(s);
  const int64_t N = s->c.N;
  out->E_int = o[0];
  out->E_kin = o[1];
  out->E = o[0] + o[1];
  out->P[0] = o[2]; out->P[1] = o[3]; out->P[2] = o[4];
  out->T_kin = N > 1 ? 2.0 * o[1] / (3.0 * (double)(N - 1) * s->c.kB) : 0.0;
  out->T_int = N > 0 ? o[5] / (double)N : 0.0;
  out->eps_min = N > 0 ? o[6] : 0.0;
  out->n_pairs = (int64_t)cnt[0];
  out->n_accept = (int64_t)cnt[1];
  out->n_reject_bound = (int64_t)cnt[2];
  out->n_reject_metropolis = (int64_t)cnt[3];
  out->fd_step = s->fd_step;
  out->vv_step = s->vv_step;
  out->status = st;
  return st;
}

int sdpd_set_fd_step(sdpd_t* s, int64_t v) {
  if (!s || v < 0) return SDPD_ERR_INVALID_ARG;
  s->fd_step = v;
  if (s->ws) {
    if (use_device(s) != SDPD_OK) return SDPD_ERR_CUDA;
    launch_set_sweep(s->w, (unsigned long long)v, s->stream);
    s->launches += 1;
    return launch_status();
  }
  return SDPD_OK;
}

int64_t sdpd_get_fd_step(const sdpd_t* s) { return s ? s->fd_step : -1; }

int sdpd_reset_counters(sdpd_t* s) {
  if (!s) return SDPD_ERR_INVALID_ARG;
  if (!s->ws) return SDPD_ERR_NO_WORKSPACE;
  if (use_device(s) != SDPD_OK) return SDPD_ERR_CUDA;
  return cuda_ok(cudaMemsetAsync(s->w.counters, 0, 4 * 8, s->stream));
}

int64_t sdpd_kernel_launches(const sdpd_t* s) { return s ? s->launches : -1; }

int sdpd_enable_stage_timing(sdpd_t* s, int on) {
  if (!s) return SDPD_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return SDPD_ERR_CUDA;
  drain_events(s);
  s->timing = on != 0;
  for (int k = 0; k < SDPD_NSTAGES; ++k) { s->stage_ms[k] = 0.0; s->stage_launches[k] = 0; }
  return SDPD_OK;
}

int sdpd_stage_times(sdpd_t* s, double* ms, int64_t* launches, int n) {
  if (!s || n < 0 || n > SDPD_NSTAGES) return SDPD_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return SDPD_ERR_CUDA;
  drain_events(s);
  for (int k = 0; k < n; ++k) {
    if (ms) ms[k] = s->stage_ms[k];
    if (launches) launches[k] = s->stage_launches[k];
  }
  return SDPD_OK;
}

}  // extern "C"

namespace {

// What the autotuners save before their trial steps and put back after:
// the state (in id order, in the staging buffers that the load path reads),
// the host step counters and the device pair counters.
struct SavedHandle {
  unsigned long long counters[4];
  int64_t fd_step, vv_step, launches;
  bool timing;
};

int save_handle(sdpd_handle* s, SavedHandle* sv) {
  cudaStream_t st = s->stream;
  if (s->prm.precision == SDPD_MIXED) launch_unload<Mixed>(s->c, s->w, s->cur, st);
  else launch_unload<Fp64>(s->c, s->w, s->cur, st);
  if (cudaMemcpyAsync(sv->counters, s->w.counters, sizeof(sv->counters), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SDPD_ERR_CUDA;
  sv->fd_step = s->fd_step;
  sv->vv_step = s->vv_step;
  sv->launches = s->launches;
  sv->timing = s->timing;
  s->timing = false;
  return SDPD_OK;
}

// the saved state loaded again (bin, sort, density) with its step counters
void reload_handle(sdpd_handle* s, const SavedHandle& sv) {
  if (s->prm.precision == SDPD_MIXED) do_load<Mixed>(s);
  else do_load<Fp64>(s);
  launch_set_sweep(s->w, (unsigned long long)sv.fd_step, s->stream);
  s->fd_step = sv.fd_step;
  s->vv_step = sv.vv_step;
}

// the device counters and status put back; synchronising (the host copy of
// the counters must outlive the transfer)
int finish_restore(sdpd_handle* s, const SavedHandle& sv) {
  int e = cuda_ok(cudaMemcpyAsync(s->w.counters, sv.counters, sizeof(sv.counters), cudaMemcpyHostToDevice, s->stream));
  e |= cuda_ok(cudaMemsetAsync(s->w.status, 0, 8, s->stream));
  s->launches = sv.launches;
  s->timing = sv.timing;
  if (e) return SDPD_ERR_CUDA;
  return sdpd_sync(s);
}

}  // namespace

extern "C" {

int sdpd_get_tuning(const sdpd_t* s, sdpd_tuning* out) {
  if (!s || !out) return SDPD_ERR_INVALID_ARG;
  out->fd_variant = s->c.fd_variant;
  out->pair_threads = s->c.pair_threads;
  return SDPD_OK;
}

int sdpd_set_tuning(sdpd_t* s, const sdpd_tuning* t) {
  if (!s || !t) return SDPD_ERR_INVALID_ARG;
  const int v = t->fd_variant < 0 ? fd_default_variant(sweep_float(s)) : t->fd_variant;
  const int pt = t->pair_threads == 0 ? 128 : t->pair_threads;
  if (v >= kFdVariants || !fd_variant_fits(sweep_float(s), v) || !pair_threads_ok(pt))
    return SDPD_ERR_INVALID_ARG;
  s->c.fd_variant = v;
  s->c.pair_threads = pt;
  return SDPD_OK;
}

int sdpd_autotune(sdpd_t* s, double dt, int64_t steps, uint64_t seed, sdpd_tuning* best, double* ms_per_step) {
  if (!s || !(dt > 0) || !isfinite(dt) || steps < 1 || steps > 1000) return SDPD_ERR_INVALID_ARG;
  if (!s->ws) return SDPD_ERR_NO_WORKSPACE;
  if (!s->has_state) return SDPD_ERR_NO_STATE;
  int e = sdpd_sync(s);
  if (e) return e;
  const bool mixed = s->prm.precision == SDPD_MIXED;
  cudaStream_t st = s->stream;
  SavedHandle sv;
  e = save_handle(s, &sv);
  if (e) return e;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
    if (ev[0]) cudaEventDestroy(ev[0]);
    s->timing = sv.timing;
    return SDPD_ERR_CUDA;
  }
  // time per step of one candidate; infinity when it failed
  auto trial = [&](int v, int pt) -> double {
    s->c.fd_variant = v;
    s->c.pair_threads = pt;
    reload_handle(s, sv);
    if (mixed) do_steps<Mixed>(s, dt, 1, seed);
    else do_steps<Fp64>(s, dt, 1, seed);
    cudaEventRecord(ev[0], st);
    if (mixed) do_steps<Mixed>(s, dt, steps, seed);
    else do_steps<Fp64>(s, dt, steps, seed);
    cudaEventRecord(ev[1], st);
    float ms = 0.0f;
    if (sdpd_sync(s) != SDPD_OK || cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) {
      cudaGetLastError();
      cudaMemsetAsync(s->w.status, 0, 8, st);
      return INFINITY;
    }
    return (double)ms / (double)steps;
  };
  const int v0 = s->c.fd_variant, t0 = s->c.pair_threads;
  int bv = v0, bt = 128;
  double bms = INFINITY;
  for (int v = 0; v < kFdVariants; ++v) {
    if (!fd_variant_fits(sweep_float(s), v)) continue;
    const double ms = trial(v, 128);
    if (ms < bms) { bms = ms; bv = v; }
  }
  for (int pt : {32, 64}) {
    const double ms = trial(bv, pt);
    if (ms < bms) { bms = ms; bt = pt; }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (!isfinite(bms)) { bv = v0; bt = t0; }
  s->c.fd_variant = bv;
  s->c.pair_threads = bt;
  reload_handle(s, sv);  // back to the state and counters the call started from
  e = finish_restore(s, sv);
  if (e) return e;
  if (best) { best->fd_variant = bv; best->pair_threads = bt; }
  if (ms_per_step) *ms_per_step = bms;
  return isfinite(bms) ? SDPD_OK : SDPD_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Gradients of the conservative dynamics (reverse mode, float64 handles)
// ---------------------------------------------------------------------------
namespace {

// The tape (caller memory): scratch of the reverse pass; the increments of
// every step's sweep (momenta [N][3], then energies [N], id order); the
// sorted momenta and energies before the current sweep; then stored states
// in id order (q [N][3], p [N][3], eps [N]): the checkpoints at steps 0,
// every, 2 every, ... below nsteps, the final state, and the every - 1
// states of the segment being replayed.
struct Tape {
  D4* vs4;
  double *A, *Sbar, *Sbar2, *qbar, *pbar, *thbar, *partial, *sums, *incr, *pre, *states;
  int64_t n_ckpt, n_seg, stride, N;
  double* ckpt(int64_t k) const { return states + k * stride; }
  double* final_state() const { return ckpt(n_ckpt); }
  double* seg(int64_t j) const { return ckpt(n_ckpt + 1 + j); }
  double* dp(int64_t step) const { return incr + step * 4 * N; }
  double* de(int64_t step) const { return incr + step * 4 * N + 3 * N; }
};

size_t tape_layout(int64_t N, int64_t nsteps, int64_t every, char* base, Tape* t) {
  const size_t n = (size_t)(N > 0 ? N : 1);
  Layout L;
  auto at = [&](size_t bytes) -> void* { return base ? base + L.take(bytes) : (L.take(bytes), nullptr); };
  t->N = N;
  t->vs4 = (D4*)at(n * sizeof(D4));
  t->A = (double*)at(n * 8);
  t->Sbar = (double*)at(n * 8);
  t->Sbar2 = (double*)at(n * 8);
  t->qbar = (double*)at(3 * n * 8);
  t->pbar = (double*)at(3 * n * 8);
  t->thbar = (double*)at(3 * n * 8);
  t->partial = (double*)at(adj_sum_partial_doubles() * 8);
  t->sums = (double*)at(4 * 8);
  t->incr = (double*)at((size_t)(nsteps > 0 ? nsteps : 1) * 4 * n * 8);
  t->pre = (double*)at(4 * n * 8);
  t->n_ckpt = (nsteps + every - 1) / every;
  t->n_seg = nsteps > 0 ? std::min<int64_t>(every, nsteps) - 1 : 0;
  t->stride = 7 * (int64_t)n;
  t->states = (double*)at((size_t)(t->n_ckpt + 1 + t->n_seg) * (size_t)t->stride * 8);
  return L.off;
}

bool tape_sizes_ok(int64_t nsteps, int64_t every) {
  return nsteps >= 0 && every >= 1 && nsteps <= (int64_t)1 << 40 && every <= (int64_t)1 << 40;
}

// copy the current state, in id order, into a tape slot
void store_state(sdpd_handle* s, double* slot) {
  Workspace w = s->w;
  w.io_q = slot;
  w.io_p = slot + 3 * s->c.N;
  w.io_e = slot + 6 * s->c.N;
  launch_unload<Fp64>(s->c, w, s->cur, s->stream);
  s->launches += 1;
}

// load a tape slot as the current state: bin, sort, density (eps kept)
void load_state(sdpd_handle* s, const double* slot) {
  Workspace w = s->w;
  w.io_q = (double*)slot;
  w.io_p = (double*)slot + 3 * s->c.N;
  w.io_e = (double*)slot + 6 * s->c.N;
  launch_load<Fp64>(s->c, w, s->stream);
  launch_sort<Fp64>(s->c, s->w, 0, s->stream);
  s->cur = 1;
  launch_density<Fp64>(s->c, s->w, s->cur, 0, nullptr, s->stream);
  s->launches += 7;
  s->sched_valid = false;
}

int check_adjoint_handle(sdpd_handle* s) {
  if (!s) return SDPD_ERR_INVALID_ARG;
  if (!s->ws) return SDPD_ERR_NO_WORKSPACE;
  if (s->prm.precision != SDPD_FP64 || s->prm.fd_only) return SDPD_ERR_INVALID_ARG;
  if (use_device(s) != SDPD_OK) return SDPD_ERR_CUDA;
  return SDPD_OK;
}

}  // namespace

extern "C" {

size_t sdpd_tape_bytes(const sdpd_t* s, int64_t nsteps, int64_t every) {
  if (!s || !tape_sizes_ok(nsteps, every)) return 0;
  Tape t;
  return tape_layout(s->c.N, nsteps, every, nullptr, &t);
}

int sdpd_vv_record(sdpd_t* s, double dt, int64_t nsteps, int64_t every, uint64_t seed, void* tape,
                   size_t tape_bytes) {
  int e = check_adjoint_handle(s);
  if (e) return e;
  if (!s->has_state) return SDPD_ERR_NO_STATE;
  if (!(dt > 0) || !isfinite(dt) || !tape_sizes_ok(nsteps, every)) return SDPD_ERR_INVALID_ARG;
  Tape t;
  if (!tape || ((uintptr_t)tape % kAlign) != 0 || tape_bytes < tape_layout(s->c.N, nsteps, every, nullptr, &t))
    return SDPD_ERR_INVALID_ARG;
  tape_layout(s->c.N, nsteps, every, (char*)tape, &t);
  s->rec.tape = nullptr;
  const int theta = s->prm.theta < 1 ? 1 : s->prm.theta;
  const size_t b1 = (size_t)s->c.N * 8;
  for (int64_t n = 0; n < nsteps; ++n) {
    if (n % every == 0) store_state(s, t.ckpt(n / every));
    vv_step<Fp64>(s, dt);
    // the sweep of this step, frozen: its increments are stored and the
    // state becomes before + increment (zero increments without a sweep)
    if (s->c.N > 0) {
      e = SDPD_OK;
      e |= cuda_ok(cudaMemcpyAsync(t.pre, s->w.px[s->cur], b1, cudaMemcpyDeviceToDevice, s->stream));
      e |= cuda_ok(cudaMemcpyAsync(t.pre + s->c.N, s->w.py[s->cur], b1, cudaMemcpyDeviceToDevice, s->stream));
      e |= cuda_ok(cudaMemcpyAsync(t.pre + 2 * s->c.N, s->w.pz[s->cur], b1, cudaMemcpyDeviceToDevice, s->stream));
      e |= cuda_ok(cudaMemcpyAsync(t.pre + 3 * s->c.N, s->w.eps[s->cur], b1, cudaMemcpyDeviceToDevice, s->stream));
      if (e) return SDPD_ERR_CUDA;
    }
    if (sweep_due(s)) fd_sweep_step<Fp64>(s, theta * dt, seed);
    launch_adj_freeze(s->c, s->w, s->cur, t.pre, t.dp(n), t.de(n), s->stream);
    s->launches += 1;
  }
  store_state(s, t.final_state());
  e = launch_status();
  if (e) return e;
  s->rec.tape = tape;
  s->rec.bytes = tape_bytes;
  s->rec.nsteps = nsteps;
  s->rec.every = every;
  s->rec.dt = dt;
  return SDPD_OK;
}

int sdpd_vv_replay(sdpd_t* s, const void* tape, size_t tape_bytes) {
  int e = check_adjoint_handle(s);
  if (e) return e;
  if (!s->has_state) return SDPD_ERR_NO_STATE;
  if (!tape || tape != s->rec.tape || tape_bytes != s->rec.bytes) return SDPD_ERR_INVALID_ARG;
  Tape t;
  tape_layout(s->c.N, s->rec.nsteps, s->rec.every, (char*)tape, &t);
  for (int64_t n = 0; n < s->rec.nsteps; ++n) {
    vv_step<Fp64>(s, s->rec.dt);
    launch_adj_increment(s->c, s->w, s->cur, t.dp(n), t.de(n), s->stream);
    s->launches += 1;
  }
  return launch_status();
}

int sdpd_tape_increments(sdpd_t* s, const void* tape, size_t tape_bytes, int64_t step, double* dp, double* deps) {
  int e = check_adjoint_handle(s);
  if (e) return e;
  if (!tape || tape != s->rec.tape || tape_bytes != s->rec.bytes || step < 0 || step >= s->rec.nsteps)
    return SDPD_ERR_INVALID_ARG;
  if (s->c.N > 0 && (!dp || !deps)) return SDPD_ERR_INVALID_ARG;
  Tape t;
  tape_layout(s->c.N, s->rec.nsteps, s->rec.every, (char*)tape, &t);
  const size_t b1 = (size_t)s->c.N * 8;
  if (s->c.N == 0) return SDPD_OK;
  e = cuda_ok(cudaMemcpyAsync(dp, t.dp(step), 3 * b1, cudaMemcpyDeviceToDevice, s->stream));
  e |= cuda_ok(cudaMemcpyAsync(deps, t.de(step), b1, cudaMemcpyDeviceToDevice, s->stream));
  return e ? SDPD_ERR_CUDA : SDPD_OK;
}

int sdpd_vv_adjoint(sdpd_t* s, void* tape, size_t tape_bytes, const double* gq, const double* gp,
                    const double* geps, double* gq0, double* gp0, double* geps0, double gtheta[3]) {
  int e = check_adjoint_handle(s);
  if (e) return e;
  if (!tape || tape != s->rec.tape || tape_bytes != s->rec.bytes) return SDPD_ERR_INVALID_ARG;
  const int64_t N = s->c.N;
  if (!gtheta || (N > 0 && (!gq0 || !gp0 || !geps0))) return SDPD_ERR_INVALID_ARG;
  const int64_t ns = s->rec.nsteps, every = s->rec.every;
  const double dt = s->rec.dt;
  Tape t;
  tape_layout(N, ns, every, (char*)tape, &t);
  const Consts& c = s->c;
  cudaStream_t st = s->stream;
  const size_t b1 = (size_t)N * 8, b3 = 3 * b1;
  e = SDPD_OK;
  if (N > 0) {
    e |= cuda_ok(gq ? cudaMemcpyAsync(t.qbar, gq, b3, cudaMemcpyDeviceToDevice, st) : cudaMemsetAsync(t.qbar, 0, b3, st));
    e |= cuda_ok(gp ? cudaMemcpyAsync(t.pbar, gp, b3, cudaMemcpyDeviceToDevice, st) : cudaMemsetAsync(t.pbar, 0, b3, st));
    e |= cuda_ok(cudaMemsetAsync(t.Sbar, 0, b1, st));
    e |= cuda_ok(cudaMemsetAsync(t.thbar, 0, b3, st));
  }
  if (e) return SDPD_ERR_CUDA;
  // Positions k = n .. 0 (states after the frozen increments of step k - 1).
  // The kicks around position k (the second of step k - 1, the first of
  // step k) both pull back along (dt/2) pbar_k, so each position is visited
  // once; their entropies differ (S_{k-1} and S_k, the sweep changed the
  // energies in between).
  int64_t seg_loaded = -1;
  // entropy cotangents of the step ending at the current position (started
  // there) and of the step starting there (completed there)
  double* Sbar_cur = t.Sbar;
  double* Sbar_prev = t.Sbar2;
  for (int64_t k = ns; k >= 0; --k) {
    if (k == ns) {
      StageTimer tm(s, 6, 7);
      load_state(s, t.final_state());
    } else if (k % every == 0) {
      StageTimer tm(s, 6, 7);
      load_state(s, t.ckpt(k / every));
    } else {
      const int64_t sg = k / every, k0 = sg * every;
      if (sg != seg_loaded) {  // replay the segment from its checkpoint
        {
          StageTimer tm(s, 6, 7);
          load_state(s, t.ckpt(sg));
        }
        const int64_t k1 = std::min(k0 + every, ns);
        for (int64_t j = k0 + 1; j < k1; ++j) {  // step j - 1, its sweep frozen
          vv_step<Fp64>(s, dt);
          s->vv_step--;
          launch_adj_increment(c, s->w, s->cur, t.dp(j - 1), t.de(j - 1), st);
          s->launches += 1;
          store_state(s, t.seg(j - k0 - 1));
        }
        seg_loaded = sg;
      }
      StageTimer tm(s, 6, 7);
      load_state(s, t.seg(k - k0 - 1));
    }
    // the first kick of step k (k < n) and the second of step k - 1 (k > 0)
    // both pull back along (dt/2) pbar
    const bool kick1 = k < ns, kick2 = k > 0;
    if (kick1 || kick2) {
      {
        StageTimer tm(s, 9, 1);
        launch_adj_gather(c, s->w, s->cur, t.pbar, 0.5 * dt, t.vs4, st);
      }
      StageTimer tm(s, 7, 1);
      launch_adj_pairsum(c, s->w, s->cur, 0, t.vs4, t.A, st);
    }
    {
      StageTimer tm(s, 9, 1);
      launch_adj_mid_step(c, s->w, s->cur, (kick1 || kick2) ? t.A : nullptr, kick1, kick2,
                          kick2 ? t.de(k - 1) : nullptr, Sbar_cur, Sbar_prev, k == ns ? geps : nullptr,
                          k == 0 ? geps0 : nullptr, t.vs4, t.thbar, st);
    }
    {
      StageTimer tm(s, 8, 1);
      launch_adj_back(c, s->w, s->cur, (kick1 || kick2) ? 0 : 2, 1.0, t.vs4, 1, t.qbar, t.thbar, st);
    }
    if (k > 0) {
      StageTimer tm(s, 9, 1);
      launch_adj_axpy(3 * N, dt / c.m, t.qbar, t.pbar, st);
    }
    std::swap(Sbar_cur, Sbar_prev);
    s->launches += ((kick1 || kick2) ? 2 : 0) + 2 + (k > 0 ? 1 : 0);
  }
  if (N > 0) {
    e |= cuda_ok(cudaMemcpyAsync(gq0, t.qbar, b3, cudaMemcpyDeviceToDevice, st));
    e |= cuda_ok(cudaMemcpyAsync(gp0, t.pbar, b3, cudaMemcpyDeviceToDevice, st));
  }
  launch_adj_sum(t.thbar, N, 3, t.partial, t.sums, st);
  s->launches += 2;
  double th[3] = {0.0, 0.0, 0.0};
  e |= cuda_ok(cudaMemcpyAsync(th, t.sums, 3 * 8, cudaMemcpyDeviceToHost, st));
  // leave the handle at the recorded final state
  load_state(s, t.final_state());
  if (e) return SDPD_ERR_CUDA;
  e = sdpd_sync(s);
  for (int k = 0; k < 3; ++k) gtheta[k] = th[k];
  return e;
}

int sdpd_virial(sdpd_t* s, double* value, double* gq, double* gp, double* geps, double gtheta[3]) {
  int e = check_adjoint_handle(s);
  if (e) return e;
  if (!s->has_state) return SDPD_ERR_NO_STATE;
  const bool grad = gq || gp || geps;
  if (!value || (grad && (!gq || !gp || !geps || !gtheta))) return SDPD_ERR_INVALID_ARG;
  const Consts& c = s->c;
  cudaStream_t st = s->stream;
  const int other = 1 - s->cur;
  // scratch: the sort target of the next step and the id-order staging
  D4* vs4 = (D4*)s->w.q4[other];
  double* A = (double*)s->w.rho[other];
  double* val_id = s->w.io_e;
  double* thbar = s->w.io_q;
  double* sums = s->w.obs + 8;  // slots 8..11 of the observables' output block
  const double wt = 1.0 / (3.0 * c.L[0] * c.L[1] * c.L[2]);
  launch_adj_pairsum(c, s->w, s->cur, 1, vs4, A, st);
  launch_adj_mid_virial(c, s->w, s->cur, A, wt, vs4, val_id, grad ? gp : nullptr, geps, thbar, st);
  if (grad) launch_adj_back(c, s->w, s->cur, 1, wt, vs4, 0, gq, thbar, st);
  launch_adj_sum(val_id, c.N, 1, (double*)s->w.obs_partial, sums, st);
  if (grad) launch_adj_sum(thbar, c.N, 3, (double*)s->w.obs_partial, sums + 1, st);
  s->launches += 4 + (grad ? 3 : 0);
  double out[4] = {0.0, 0.0, 0.0, 0.0};
  if (cudaMemcpyAsync(out, sums, 4 * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return SDPD_ERR_CUDA;
  e = sdpd_sync(s);
  *value = out[0];
  if (grad)
    for (int k = 0; k < 3; ++k) gtheta[k] = out[1 + k];
  return e;
}

int sdpd_energy_histogram(sdpd_t* s, double lo, double hi, int nbins, double scale, unsigned long long* counts) {
  if (!s) return SDPD_ERR_INVALID_ARG;
  if (!s->ws) return SDPD_ERR_NO_WORKSPACE;
  if (!s->has_state) return SDPD_ERR_NO_STATE;
  if (!counts || nbins < 1 || nbins > 4096 || !isfinite(lo) || !isfinite(hi) || !(hi > lo) || !isfinite(scale))
    return SDPD_ERR_INVALID_ARG;
  if (use_device(s) != SDPD_OK) return SDPD_ERR_CUDA;
  launch_energy_hist(s->c, s->w, s->cur, lo, hi, nbins, scale, counts, s->stream);
  s->launches += s->c.N > 0 ? 1 : 0;
  return launch_status();
}

}  // extern "C"

namespace {

// Body of sdpd_debug_get.  Every host staging buffer is allocated after the
// capacity check, and every copy into one is synchronised before it is read
// or goes out of scope.
int debug_get(sdpd_handle* s, int what, void* dst, int64_t cap, int64_t* count) {
  const int64_t N = s->c.N;
  const bool mixed = s->prm.precision == SDPD_MIXED;
  cudaStream_t st = s->stream;
  const int cur = s->cur;
  std::vector<int32_t> ids;
  // ids in storage order, copied asynchronously; the caller synchronises
  auto fetch_ids = [&]() -> bool {
    ids.resize((size_t)N);
    return N == 0 || cudaMemcpyAsync(ids.data(), s->w.id[cur], (size_t)N * 4, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  };
  switch (what) {
    case SDPD_DEBUG_ORDER: {
      if (cap < N) return SDPD_ERR_INVALID_ARG;
      if (!fetch_ids()) return SDPD_ERR_CUDA;
      if (cudaStreamSynchronize(st) != cudaSuccess) return SDPD_ERR_CUDA;
      int64_t* o = (int64_t*)dst;
      for (int64_t t = 0; t < N; ++t) o[t] = ids[(size_t)t];
      if (count) *count = N;
      return sdpd_sync(s);
    }
    case SDPD_DEBUG_CELLS: {
      if (cap < N) return SDPD_ERR_INVALID_ARG;
      const size_t rec = mixed ? 16 : 32;
      std::vector<unsigned char> q4((size_t)N * rec);
      if (!fetch_ids()) return SDPD_ERR_CUDA;
      if (N > 0 && cudaMemcpyAsync(q4.data(), s->w.q4[cur], (size_t)N * rec, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        cudaStreamSynchronize(st);
        return SDPD_ERR_CUDA;
      }
      if (cudaStreamSynchronize(st) != cudaSuccess) return SDPD_ERR_CUDA;
      int32_t* o = (int32_t*)dst;
      for (int64_t t = 0; t < N; ++t) {
        uint32_t cb;
        if (mixed) {
          memcpy(&cb, &q4[(size_t)t * rec + 12], 4);
        } else {
          double w;
          memcpy(&w, &q4[(size_t)t * rec + 24], 8);
          cb = (uint32_t)w;
        }
        int cx, cy, cz;
        unpack_cell(cb, cx, cy, cz);
        const int64_t k = ids[(size_t)t];
        o[3 * k] = cx; o[3 * k + 1] = cy; o[3 * k + 2] = cz;
      }
      if (count) *count = N;
      return sdpd_sync(s);
    }
    case SDPD_DEBUG_RHO: {
      if (cap < N) return SDPD_ERR_INVALID_ARG;
      double* o = (double*)dst;
      if (mixed) {
        std::vector<float> r((size_t)N);
        if (!fetch_ids()) return SDPD_ERR_CUDA;
        if (N > 0 && cudaMemcpyAsync(r.data(), s->w.rho[cur], (size_t)N * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
          cudaStreamSynchronize(st);
          return SDPD_ERR_CUDA;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) return SDPD_ERR_CUDA;
        for (int64_t t = 0; t < N; ++t) o[ids[(size_t)t]] = r[(size_t)t];
      } else {
        std::vector<double> r((size_t)N);
        if (!fetch_ids()) return SDPD_ERR_CUDA;
        if (N > 0 && cudaMemcpyAsync(r.data(), s->w.rho[cur], (size_t)N * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
          cudaStreamSynchronize(st);
          return SDPD_ERR_CUDA;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) return SDPD_ERR_CUDA;
        for (int64_t t = 0; t < N; ++t) o[ids[(size_t)t]] = r[(size_t)t];
      }
      if (count) *count = N;
      return sdpd_sync(s);
    }
    case SDPD_DEBUG_FORCE: {
      if (cap < 3 * N) return SDPD_ERR_INVALID_ARG;
      if (mixed) launch_force<Mixed>(s->c, s->w, cur, 0.0, 0.0, s->w.io_p, st);
      else launch_force<Fp64>(s->c, s->w, cur, 0.0, 0.0, s->w.io_p, st);
      s->launches += 2;
      if (N > 0 && cudaMemcpyAsync(dst, s->w.io_p, (size_t)N * 24, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SDPD_ERR_CUDA;
      if (count) *count = 3 * N;
      return sdpd_sync(s);
    }
    case SDPD_DEBUG_NCOUNT: {
      if (cap < N) return SDPD_ERR_INVALID_ARG;
      if (mixed) launch_density<Mixed>(s->c, s->w, cur, 0, (int32_t*)s->w.io_q, st);
      else launch_density<Fp64>(s->c, s->w, cur, 0, (int32_t*)s->w.io_q, st);
      s->launches += 1;
      if (N > 0 && cudaMemcpyAsync(dst, s->w.io_q, (size_t)N * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SDPD_ERR_CUDA;
      if (count) *count = N;
      return sdpd_sync(s);
    }
    case SDPD_DEBUG_PAIRS: {
      if (!s->w.pair_recs) return SDPD_ERR_INVALID_ARG;
      unsigned long long n = 0;
      if (cudaMemcpyAsync(&n, s->w.pair_rec_count, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return SDPD_ERR_CUDA;
      if (cudaStreamSynchronize(st) != cudaSuccess) return SDPD_ERR_CUDA;
      int64_t m = std::min<int64_t>((int64_t)n, s->w.pair_rec_cap);
      if (cap < m) return SDPD_ERR_INVALID_ARG;
      if (m > 0 && cudaMemcpyAsync(dst, s->w.pair_recs, (size_t)m * sizeof(sdpd_pair_rec), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SDPD_ERR_CUDA;
      if (count) *count = m;
      int r = sdpd_sync(s);
      if (r == SDPD_OK && (int64_t)n > s->w.pair_rec_cap) return SDPD_ERR_CAPACITY;
      return r;
    }
    case SDPD_DEBUG_BIG: {
      if (cap < 8) return SDPD_ERR_INVALID_ARG;
      if (cudaMemcpyAsync(dst, s->w.big_count, 8 * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SDPD_ERR_CUDA;
      if (count) *count = 8;
      return sdpd_sync(s);
    }
    default:
      return SDPD_ERR_INVALID_ARG;
  }
}

}  // namespace

extern "C" {

int sdpd_debug_get(sdpd_t* s, int what, void* dst, int64_t cap, int64_t* count) {
  if (!s || !dst) return SDPD_ERR_INVALID_ARG;
  if (!s->ws) return SDPD_ERR_NO_WORKSPACE;
  if (use_device(s) != SDPD_OK) return SDPD_ERR_CUDA;
  if (!s->has_state) return SDPD_ERR_NO_STATE;
  if (count) *count = 0;
  try {
    return debug_get(s, what, dst, cap, count);
  } catch (const std::bad_alloc&) {
    cudaStreamSynchronize(s->stream);
    return SDPD_ERR_HOST_MEMORY;
  }
}

// ---------------------------------------------------------------------------
// Ensembles of independent systems stepped by one CUDA graph.
// ---------------------------------------------------------------------------
// longest graph replay unit (steps) of an ensemble: lcm(2, theta_i)
constexpr int64_t kMaxEnsembleUnit = 64;

struct sdpd_ensemble {
  std::vector<sdpd_handle*> m;
  cudaStream_t stream;
  cudaEvent_t fork;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool own_stream;
  double dt;
  std::vector<uint64_t> seeds;
  int64_t launches_per_unit;
  int64_t unit;                  // steps per graph replay: lcm of 2 and the members' theta
  std::vector<int64_t> phase;    // members' vv_step mod theta when the graph was captured
  std::vector<int> shape;        // members' state buffer and launch shapes at capture
};

namespace {

void member_steps(sdpd_handle* h, double dt, int64_t n, uint64_t seed) {
  if (h->prm.precision == SDPD_MIXED) do_steps<Mixed>(h, dt, n, seed);
  else do_steps<Fp64>(h, dt, n, seed);
}

// Enqueue nsteps steps of every member on its own stream, forked from and
// joined back into the ensemble stream.
void ensemble_enqueue(sdpd_ensemble* e, double dt, int64_t nsteps, const uint64_t* seeds) {
  cudaEventRecord(e->fork, e->stream);
  for (size_t i = 0; i < e->m.size(); ++i) {
    sdpd_handle* h = e->m[i];
    cudaStreamWaitEvent(h->stream, e->fork, 0);
    member_steps(h, dt, nsteps, seeds[i]);
    cudaEventRecord(e->join[i], h->stream);
    cudaStreamWaitEvent(e->stream, e->join[i], 0);
  }
}

// Make `to` wait for the work already enqueued on `from`.
int order_streams(cudaStream_t from, cudaStream_t to) {
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return SDPD_ERR_CUDA;
  int st = cuda_ok(cudaEventRecord(ev, from));
  st |= cuda_ok(cudaStreamWaitEvent(to, ev, 0));
  cudaEventDestroy(ev);
  return st ? SDPD_ERR_CUDA : SDPD_OK;
}

}  // namespace

int sdpd_ensemble_create(sdpd_t* const* members, int n, void* stream, sdpd_ens_t** out) {
  if (!out) return SDPD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!members || n < 1) return SDPD_ERR_INVALID_ARG;
  sdpd_ensemble* e = new (std::nothrow) sdpd_ensemble();
  if (!e) return SDPD_ERR_INVALID_ARG;
  e->stream = (cudaStream_t)stream;
  e->own_stream = false;
  e->graph = nullptr;
  e->exec = nullptr;
  e->dt = 0.0;
  try {
    e->m.reserve((size_t)n);
    e->join.assign((size_t)n, nullptr);
  } catch (const std::bad_alloc&) {
    delete e;
    return SDPD_ERR_HOST_MEMORY;
  }
  for (int i = 0; i < n; ++i) {
    sdpd_handle* h = members[i];
    if (!h || !h->ws || !h->has_state || h->timing || h->w.pair_recs || h->stream == e->stream) {
      delete e;
      return !h || h->ws ? SDPD_ERR_INVALID_ARG : SDPD_ERR_NO_WORKSPACE;
    }
    // one graph runs on one device: every member's workspace on the first's
    if (h->device != members[0]->device) { delete e; return SDPD_ERR_INVALID_ARG; }
    for (int j = 0; j < i; ++j)
      if (members[j] == h) { delete e; return SDPD_ERR_INVALID_ARG; }
    e->m.push_back(h);
  }
  e->unit = 2;
  for (sdpd_handle* h : e->m) {
    const int64_t th = std::max(1, h->prm.theta);
    e->unit = e->unit / std::gcd(e->unit, th) * th;
    if (e->unit > kMaxEnsembleUnit) { delete e; return SDPD_ERR_INVALID_ARG; }
  }
  if (use_device(e->m[0]) != SDPD_OK || cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) != cudaSuccess) {
    delete e;
    return SDPD_ERR_CUDA;
  }
  if (!e->stream) {  // a stream of the ensemble's own (the legacy default stream cannot be captured)
    if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaEventDestroy(e->fork);
      delete e;
      return SDPD_ERR_CUDA;
    }
    e->own_stream = true;
  }
  for (int i = 0; i < n; ++i) {
    if (cudaEventCreateWithFlags(&e->join[(size_t)i], cudaEventDisableTiming) != cudaSuccess) {
      e->join[(size_t)i] = nullptr;
      sdpd_ensemble_destroy(e);
      return SDPD_ERR_CUDA;
    }
  }
  *out = e;
  return SDPD_OK;
}

int sdpd_ensemble_step(sdpd_ens_t* e, double dt, int64_t nsteps, const uint64_t* seeds) {
  if (!e || !seeds || !(dt > 0) || !isfinite(dt) || nsteps < 0) return SDPD_ERR_INVALID_ARG;
  if (use_device(e->m[0]) != SDPD_OK) return SDPD_ERR_CUDA;
  // the ensemble stream waits for everything already enqueued on the members
  for (sdpd_handle* h : e->m)
    if (order_streams(h->stream, e->stream) != SDPD_OK) return SDPD_ERR_CUDA;
  const int64_t U = e->unit;
  const int64_t units = nsteps / U;
  const std::vector<uint64_t> sv(seeds, seeds + e->m.size());
  std::vector<int64_t> phase;
  std::vector<int> shape;
  for (sdpd_handle* h : e->m) {
    phase.push_back(h->vv_step % std::max(1, h->prm.theta));
    // the graph holds the buffer pointers and launch shapes of its capture
    shape.push_back(h->cur);
    shape.push_back(h->c.fd_variant);
    shape.push_back(h->c.pair_threads);
  }
  if (units > 0) {
    if (!e->exec || e->dt != dt || e->seeds != sv || e->phase != phase || e->shape != shape) {
      if (e->exec) { cudaGraphExecDestroy(e->exec); e->exec = nullptr; }
      if (e->graph) { cudaGraphDestroy(e->graph); e->graph = nullptr; }
      // capture U steps: each step's sort flips the double-buffered state,
      // so after an even number of steps every member is back in its
      // buffer, and U is a multiple of every member's theta, so the sweeps
      // fall on the same steps of every replay; host bookkeeping is
      // restored after capture
      std::vector<int> cur0;
      std::vector<int64_t> fd0, vv0, l0;
      for (sdpd_handle* h : e->m) {
        cur0.push_back(h->cur); fd0.push_back(h->fd_step); vv0.push_back(h->vv_step); l0.push_back(h->launches);
      }
      if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SDPD_ERR_CUDA;
      ensemble_enqueue(e, dt, U, seeds);
      cudaError_t ce = cudaStreamEndCapture(e->stream, &e->graph);
      e->launches_per_unit = 0;
      for (size_t i = 0; i < e->m.size(); ++i) {
        sdpd_handle* h = e->m[i];
        e->launches_per_unit += h->launches - l0[i];
        h->cur = cur0[i]; h->fd_step = fd0[i]; h->vv_step = vv0[i]; h->launches = l0[i];
      }
      if (ce != cudaSuccess || cudaGraphInstantiate(&e->exec, e->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return SDPD_ERR_CUDA;
      }
      e->dt = dt;
      e->seeds = sv;
      e->phase = phase;
      e->shape = shape;
    }
    for (int64_t u = 0; u < units; ++u)
      if (cudaGraphLaunch(e->exec, e->stream) != cudaSuccess) return SDPD_ERR_CUDA;
    for (sdpd_handle* h : e->m) {
      if (!h->prm.fd_only) h->vv_step += U * units;
      if (h->prm.scheme != SDPD_SCHEME_NONE)
        h->fd_step += h->prm.fd_only ? U * units : U / std::max(1, h->prm.theta) * units;
      h->sched_valid = h->prm.fd_only ? true : false;
    }
    const int64_t per_member = e->launches_per_unit / (int64_t)e->m.size();
    for (sdpd_handle* h : e->m) h->launches += per_member * units;
  }
  if (nsteps % U) ensemble_enqueue(e, dt, nsteps % U, seeds);
  // later calls on a member's own stream see the ensemble's work
  for (sdpd_handle* h : e->m)
    if (order_streams(e->stream, h->stream) != SDPD_OK) return SDPD_ERR_CUDA;
  return launch_status();
}

int sdpd_ensemble_autotune(sdpd_ens_t* e, double dt, int64_t steps, const uint64_t* seeds, double* ms_per_step) {
  if (!e || !(dt > 0) || !isfinite(dt) || steps < 1 || steps > 1000) return SDPD_ERR_INVALID_ARG;
  const size_t n = e->m.size();
  std::vector<uint64_t> sd(n, 0ull);
  if (seeds) sd.assign(seeds, seeds + n);
  // members' streams may still hold work of the ensemble stream
  for (sdpd_handle* h : e->m)
    if (order_streams(e->stream, h->stream) != SDPD_OK) return SDPD_ERR_CUDA;
  // 1. every member alone
  std::vector<sdpd_tuning> alone(n);
  for (size_t i = 0; i < n; ++i) {
    const int r = sdpd_autotune(e->m[i], dt, steps, sd[i], &alone[i], nullptr);
    if (r != SDPD_OK) return r;
  }
  // 2. the whole ensemble, through its graph, under candidate assignments:
  // the defaults, the shapes each member chose alone, and every colour
  // schedule given to all members; the fastest assignment is kept
  std::vector<std::vector<sdpd_tuning>> cand;
  std::vector<sdpd_tuning> dflt(n);
  for (size_t i = 0; i < n; ++i) dflt[i] = {fd_default_variant(sweep_float(e->m[i])), 128};
  cand.push_back(dflt);
  cand.push_back(alone);
  for (int v = 0; v < kFdVariants; ++v) {
    std::vector<sdpd_tuning> u(n);
    for (size_t i = 0; i < n; ++i) {
      const bool fl = sweep_float(e->m[i]);
      u[i] = {fd_variant_fits(fl, v) ? v : fd_default_variant(fl), 128};
    }
    cand.push_back(u);
  }
  std::vector<SavedHandle> sv(n);
  for (size_t i = 0; i < n; ++i) {
    const int r = save_handle(e->m[i], &sv[i]);
    if (r != SDPD_OK) {
      for (size_t k = 0; k < i; ++k) e->m[k]->timing = sv[k].timing;
      return r;
    }
  }
  const int64_t U = e->unit;
  const int64_t timed = ((steps + U - 1) / U) * U;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int err = SDPD_OK;
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) err = SDPD_ERR_CUDA;
  double bms = INFINITY;
  size_t best = 0;
  for (size_t c = 0; c < cand.size() && !err; ++c) {
    for (size_t i = 0; i < n; ++i) {
      e->m[i]->c.fd_variant = cand[c][i].fd_variant;
      e->m[i]->c.pair_threads = cand[c][i].pair_threads;
      reload_handle(e->m[i], sv[i]);
    }
    double ms = INFINITY;
    if (sdpd_ensemble_step(e, dt, U, sd.data()) == SDPD_OK) {  // capture and warm up
      cudaEventRecord(ev[0], e->stream);
      const int r = sdpd_ensemble_step(e, dt, timed, sd.data());
      cudaEventRecord(ev[1], e->stream);
      float t = 0.0f;
      bool ok = r == SDPD_OK && cudaEventSynchronize(ev[1]) == cudaSuccess &&
                cudaEventElapsedTime(&t, ev[0], ev[1]) == cudaSuccess;
      for (sdpd_handle* h : e->m) ok = (sdpd_sync(h) == SDPD_OK) && ok;
      if (ok) ms = (double)t / (double)timed;
    }
    if (!isfinite(ms)) {
      cudaGetLastError();
      for (sdpd_handle* h : e->m) cudaMemsetAsync(h->w.status, 0, 8, h->stream);
    }
    if (ms < bms) { bms = ms; best = c; }
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (!isfinite(bms)) best = 0;
  // the chosen shapes, and every member back where the call found it
  for (size_t i = 0; i < n; ++i) {
    e->m[i]->c.fd_variant = cand[best][i].fd_variant;
    e->m[i]->c.pair_threads = cand[best][i].pair_threads;
    reload_handle(e->m[i], sv[i]);
  }
  for (size_t i = 0; i < n; ++i) {
    const int r = finish_restore(e->m[i], sv[i]);
    if (!err) err = r;
  }
  if (err) return err;
  if (ms_per_step) *ms_per_step = bms;
  return isfinite(bms) ? SDPD_OK : SDPD_ERR_CUDA;
}

int64_t sdpd_ensemble_kernel_nodes(const sdpd_ens_t* e) { return e ? e->launches_per_unit : -1; }

void* sdpd_ensemble_stream(const sdpd_ens_t* e) { return e ? (void*)e->stream : nullptr; }

void sdpd_ensemble_destroy(sdpd_ens_t* e) {
  if (!e) return;
  cudaStreamSynchronize(e->stream);
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  cudaEventDestroy(e->fork);
  for (cudaEvent_t ev : e->join)
    if (ev) cudaEventDestroy(ev);
  if (e->own_stream) cudaStreamDestroy(e->stream);
  delete e;
}

void sdpd_destroy(sdpd_t* s) {
  if (!s) return;
  if (!s->ev_pending.empty()) {
    cudaStreamSynchronize(s->stream);
    drain_events(s);
  }
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  delete s;
}

}  // extern "C"
