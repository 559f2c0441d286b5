// sdpd_noalloc.cu -- the density pass for callers that cannot allocate device
// memory.  Its working memory (cell counts, cell starts, binned particle
// order) is one file-scope static device array of fixed size instead of a
// caller-bound workspace; the caller passes only the positions and the
// output.  The computation is the float64 density of the library (binning
// into cells of side >= h, 27-cell neighbour search with the periodic
// minimum image, r^2 < h^2, self term included).
#include <math.h>

#include "sdpd_internal.cuh"

namespace {

constexpr int64_t kStaticMaxN = 65536;      // particles per call
constexpr int64_t kStaticMaxCells = 65536;  // cells per call
constexpr int kMaxDevices = 64;

// scratch layout: cell_count [kStaticMaxCells], cell_start [kStaticMaxCells + 1],
// binned order [kStaticMaxN], cell of particle [kStaticMaxN], arrival slot [kStaticMaxN]
constexpr size_t kScratchInts = 2 * kStaticMaxCells + 1 + 3 * kStaticMaxN;
static __device__ __align__(256) int32_t g_noalloc_scratch[kScratchInts];

// device address of the scratch array, resolved once per device
int32_t* g_scratch_ptr[kMaxDevices] = {nullptr};

struct StaticGrid {
  int64_t N;
  int nc[3];
  int ncell;
  double L[3], halfL[3], cs[3];
  double h, h2, m, cW;
  int kernel;
};

__global__ void k_static_zero(int32_t* cnt, int ncell) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncell) cnt[c] = 0;
}

// cell of a coordinate already wrapped into [0, L)
__device__ __forceinline__ int static_cell_1d(double x, double cs, int n) {
  int c = (int)floor(__ddiv_rn(x, cs));
  return c >= n ? n - 1 : (c < 0 ? 0 : c);
}

__global__ void k_static_bin(StaticGrid g, const double* __restrict__ q, int32_t* cnt, int32_t* cell_of,
                             int32_t* slot) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int c[3];
  for (int d = 0; d < 3; ++d) c[d] = static_cell_1d(sdpd::wrap_coord(q[3 * i + d], g.L[d]), g.cs[d], g.nc[d]);
  const int lin = c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
  cell_of[i] = lin;
  slot[i] = atomicAdd(&cnt[lin], 1);
}

// exclusive scan of the cell counts by one block
__global__ void k_static_scan(int ncell, const int32_t* __restrict__ cnt, int32_t* __restrict__ start) {
  __shared__ int32_t warp_tot[32];
  const int per = (ncell + 1023) / 1024;
  const int beg = threadIdx.x * per, end = min(ncell, beg + per);
  int32_t local = 0;
  for (int i = beg; i < end; ++i) local += cnt[i];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t v = local;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int32_t t = warp_tot[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  int32_t run = v - local + (wid > 0 ? warp_tot[wid - 1] : 0);
  for (int i = beg; i < end; ++i) {
    start[i] = run;
    run += cnt[i];
  }
  if (threadIdx.x == 1023) start[ncell] = warp_tot[31];
}

__global__ void k_static_scatter(int64_t N, const int32_t* __restrict__ cell_of, const int32_t* __restrict__ slot,
                                 const int32_t* __restrict__ start, int32_t* __restrict__ order) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) order[start[cell_of[i]] + slot[i]] = (int32_t)i;
}

__device__ __forceinline__ double static_W(const StaticGrid& g, double x) {
  const double y = 1.0 - x;
  if (g.kernel == SDPD_KERNEL_LUCY) return g.cW * (1.0 + 3.0 * x) * (y * y * y);
  if (x <= 0.5) return g.cW * (1.0 - 6.0 * x * x + 6.0 * x * x * x);
  return 2.0 * g.cW * (y * y * y);
}

__global__ void k_static_density(StaticGrid g, const double* __restrict__ q, const int32_t* __restrict__ cell_of,
                                 const int32_t* __restrict__ start, const int32_t* __restrict__ order,
                                 double* __restrict__ rho) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  // coordinates wrapped periodically into [0, L), as the regular path stores them
  const double xi = sdpd::wrap_coord(q[3 * i], g.L[0]), yi = sdpd::wrap_coord(q[3 * i + 1], g.L[1]),
               zi = sdpd::wrap_coord(q[3 * i + 2], g.L[2]);
  const int lin = cell_of[i];
  const int cx = lin % g.nc[0], cy = (lin / g.nc[0]) % g.nc[1], cz = lin / (g.nc[0] * g.nc[1]);
  const double inv_h = 1.0 / g.h;
  double acc = 0.0;
  for (int oz = -1; oz <= 1; ++oz) {
    const int nz = (cz + oz + g.nc[2]) % g.nc[2];
    for (int oy = -1; oy <= 1; ++oy) {
      const int ny = (cy + oy + g.nc[1]) % g.nc[1];
      for (int ox = -1; ox <= 1; ++ox) {
        const int nx = (cx + ox + g.nc[0]) % g.nc[0];
        const int c = nx + g.nc[0] * (ny + g.nc[1] * nz);
        for (int t = start[c]; t < start[c + 1]; ++t) {
          const int j = order[t];
          if (j == i) continue;
          const double xj = sdpd::wrap_coord(q[3 * j], g.L[0]), yj = sdpd::wrap_coord(q[3 * j + 1], g.L[1]),
                       zj = sdpd::wrap_coord(q[3 * j + 2], g.L[2]);
          const double dx = sdpd::min_image(__dsub_rn(xi, xj), g.L[0], g.halfL[0]);
          const double dy = sdpd::min_image(__dsub_rn(yi, yj), g.L[1], g.halfL[1]);
          const double dz = sdpd::min_image(__dsub_rn(zi, zj), g.L[2], g.halfL[2]);
          const double r2 = sdpd::r2_of(dx, dy, dz);
          if (r2 < g.h2) acc += static_W(g, sqrt(r2) * inv_h);
        }
      }
    }
  }
  rho[i] = g.m * (g.cW + acc);
}

}  // namespace

extern "C" int sdpd_density_static(int64_t N, const double box[3], double m, double h, int kernel,
                                   const double* q, double* rho, void* stream) {
  if (!box || N < 0 || !(m > 0) || !(h > 0) || !isfinite(m) || !isfinite(h)) return SDPD_ERR_INVALID_ARG;
  if (kernel != SDPD_KERNEL_CUBIC && kernel != SDPD_KERNEL_LUCY) return SDPD_ERR_INVALID_ARG;
  if (N > kStaticMaxN) return SDPD_ERR_CAPACITY;
  if (N > 0 && (!q || !rho)) return SDPD_ERR_INVALID_ARG;
  StaticGrid g;
  g.N = N;
  int64_t ncell = 1;
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0) || !isfinite(box[d])) return SDPD_ERR_INVALID_ARG;
    double ratio = floor(box[d] / h);
    int64_t n = ratio > 1024.0 ? 1024 : (int64_t)ratio;
    n -= n % 2;
    if (n < 4) return SDPD_ERR_BOX_TOO_SMALL;
    g.nc[d] = (int)n;
    g.L[d] = box[d];
    g.halfL[d] = 0.5 * box[d];
    g.cs[d] = box[d] / (double)n;
    ncell *= n;
  }
  if (ncell > kStaticMaxCells) return SDPD_ERR_CAPACITY;
  g.ncell = (int)ncell;
  g.h = h;
  g.h2 = h * h;
  g.m = m;
  g.kernel = kernel;
  const double h3 = h * h * h;
  g.cW = kernel == SDPD_KERNEL_LUCY ? 105.0 / (16.0 * M_PI * h3) : 8.0 / (M_PI * h3);
  if (N == 0) return SDPD_OK;
  // set-up, once per device: the device address of the static array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SDPD_ERR_CUDA;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SDPD_ERR_CUDA;
    g_scratch_ptr[dev] = (int32_t*)p;
  }
  int32_t* cnt = g_scratch_ptr[dev];
  int32_t* start = cnt + kStaticMaxCells;
  int32_t* order = start + kStaticMaxCells + 1;
  int32_t* cell_of = order + kStaticMaxN;
  int32_t* slot = cell_of + kStaticMaxN;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned nbp = (unsigned)((N + 127) / 128);
  k_static_zero<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(cnt, (int)ncell);
  k_static_bin<<<nbp, 128, 0, s>>>(g, q, cnt, cell_of, slot);
  k_static_scan<<<1, 1024, 0, s>>>((int)ncell, cnt, start);
  k_static_scatter<<<nbp, 128, 0, s>>>(N, cell_of, slot, start, order);
  k_static_density<<<nbp, 128, 0, s>>>(g, q, cell_of, start, order, rho);
  return cudaGetLastError() == cudaSuccess ? SDPD_OK : SDPD_ERR_CUDA;
}
