// sdpd_sort.cu -- cell binning and the deterministic counting sort of the
// particles into Morton order of cells, ties by id; state load and unload.
//
// The sort is a bucket sort: each particle's cell was counted with an atomic
// increment when its position was (re)computed (load or drift), the counts are
// scanned into cell ranges, the particles are scattered into their cell's
// range in arrival order, and each particle's final place is its cell start
// plus the number of particles of the same cell with a smaller id.  The
// result is a pure function of (cell, id), whatever the arrival order.
#include "sdpd_internal.cuh"

namespace sdpd {

// Cell of a float64 coordinate: floor(x / cs), clamped into [0, n).
__device__ __forceinline__ int cell_of(double x, double cs, int n) {
  int c = (int)floor(__ddiv_rn(x, cs));
  return c >= n ? n - 1 : (c < 0 ? 0 : c);
}
// Cell of a fixed-point coordinate: floor(u * n / 2^32), exact.
__device__ __forceinline__ int cell_of(uint32_t u, int n) { return (int)__umulhi(u, (uint32_t)n); }


template <class P>
__global__ void k_load(Consts c, const double* __restrict__ io_q, const double* __restrict__ io_p,
                       const double* __restrict__ io_e, Arrays<P> a, typename P::Q* qdx,
                       typename P::Q* qdy, typename P::Q* qdz, const int32_t* __restrict__ mrank,
                       int32_t* key, int32_t* slot, int32_t* cell_count, int* status) {
  using R = typename P::R;
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= c.N) return;
  int cc[3];
  typename P::Q qq[3];
  for (int d = 0; d < 3; ++d) {
    double x = wrap_coord(io_q[3 * k + d], c.L[d]);
    if constexpr (P::mixed) {
      uint64_t u = (uint64_t)llrint(x * c.inv_scale[d]);
      qq[d] = (uint32_t)(u & 0xffffffffull);
      cc[d] = cell_of((uint32_t)qq[d], c.nc[d]);
    } else {
      qq[d] = x;
      cc[d] = cell_of(x, c.cs[d], c.nc[d]);
    }
  }
  qdx[k] = qq[0];
  qdy[k] = qq[1];
  qdz[k] = qq[2];
  a.px[k] = (R)io_p[3 * k];
  a.py[k] = (R)io_p[3 * k + 1];
  a.pz[k] = (R)io_p[3 * k + 2];
  double e = io_e[k];
  if (!(e > 0.0) || !isfinite(e)) atomicOr(status, kStBadEnergy);
  a.eps[k] = e;
  a.rho[k] = R(1);
  a.id[k] = (int32_t)k;
  int r = mrank[cc[0] + c.nc[0] * (cc[1] + c.nc[1] * cc[2])];
  key[k] = r;
  slot[k] = atomicAdd(&cell_count[r], 1);
}

// Exclusive scan of the cell counts in three passes (tile sums, scan of the
// tile sums in one block, tile scans); leaves the counts at zero.
constexpr int kScanTile = 2048;  // cells per tile: 256 threads x 8

__global__ void __launch_bounds__(256) k_scan_tiles(int ncell, const int32_t* __restrict__ cell_count,
                                                    int32_t* __restrict__ tile_sum) {
  __shared__ int32_t red[8];
  const int base = blockIdx.x * kScanTile + threadIdx.x * 8;
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += base + k < ncell ? cell_count[base + k] : 0;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int k = 0; k < 8; ++k) t += red[k];
    tile_sum[blockIdx.x] = t;
  }
}

// exclusive scan of up to 1024 * 32 tile sums by one block of 1024 threads
__global__ void __launch_bounds__(1024) k_scan_sums(int ntiles, int32_t* __restrict__ tile_sum, int32_t* total) {
  __shared__ int32_t warp_tot[32];
  const int per = (ntiles + 1023) / 1024;
  const int beg = threadIdx.x * per, end = min(ntiles, beg + per);
  int32_t local = 0;
  for (int i = beg; i < end; ++i) local += tile_sum[i];
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
    const int32_t n = tile_sum[i];
    tile_sum[i] = run;
    run += n;
  }
  if (threadIdx.x == 1023) *total = warp_tot[31];
}

__global__ void __launch_bounds__(256) k_scan_apply(int ncell, int32_t* __restrict__ cell_count,
                                                    int32_t* __restrict__ cell_start,
                                                    const int32_t* __restrict__ tile_sum) {
  __shared__ int32_t warp_tot[8];
  const int base = blockIdx.x * kScanTile + threadIdx.x * 8;
  int32_t v[8], s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = base + k < ncell ? cell_count[base + k] : 0;
    s += v[k];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  int32_t wbase = 0;
  for (int k = 0; k < wid; ++k) wbase += warp_tot[k];
  int32_t run = tile_sum[blockIdx.x] + wbase + incl - s;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (base + k < ncell) {
      cell_start[base + k] = run;
      cell_count[base + k] = 0;
    }
    run += v[k];
  }
}

__global__ void k_scatter(int64_t N, const int32_t* __restrict__ key, const int32_t* __restrict__ slot,
                          const int32_t* __restrict__ cell_start, const int32_t* __restrict__ id,
                          int32_t* tmp, int32_t* tmpid) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= N) return;
  int32_t pos = cell_start[key[s]] + slot[s];
  tmp[pos] = (int32_t)s;
  tmpid[pos] = id[s];
}

template <class P>
__global__ void k_gather(Consts c, const int32_t* __restrict__ tmp, const int32_t* __restrict__ tmpid,
                         const int32_t* __restrict__ key, const int32_t* __restrict__ cell_start,
                         const uint32_t* __restrict__ rcoord, const typename P::Q* __restrict__ qdx,
                         const typename P::Q* __restrict__ qdy, const typename P::Q* __restrict__ qdz,
                         Arrays<P> src, Arrays<P> dst, const uint32_t* __restrict__ xmx,
                         const uint32_t* __restrict__ xmy, const uint32_t* __restrict__ xmz,
                         float4* __restrict__ qf4) {
  using V4 = typename P::V4;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= c.N) return;
  int32_t s = tmp[t];
  int32_t myid = tmpid[t];
  int32_t r = key[s];
  int32_t beg = cell_start[r], end = cell_start[r + 1];
  int32_t rank = 0;
  for (int32_t u = beg; u < end; ++u) rank += (tmpid[u] < myid);
  int64_t d = beg + rank;
  uint32_t cb = rcoord[r];
  typename P::Q x = qdx[s], y = qdy[s], z = qdz[s];
  dst.qx[d] = x;
  dst.qy[d] = y;
  dst.qz[d] = z;
  V4 v;
  if constexpr (P::mixed) {
    int cx, cy, cz;
    unpack_cell(cb, cx, cy, cz);
    v.x = __uint2float_rn(x - xmx[cx]) * (float)c.scale[0];
    v.y = __uint2float_rn(y - xmy[cy]) * (float)c.scale[1];
    v.z = __uint2float_rn(z - xmz[cz]) * (float)c.scale[2];
  } else {
    v.x = x; v.y = y; v.z = z;
    qf4[d] = make_float4((float)x, (float)y, (float)z, 0.0f);
  }
  v.w = cellbits_to_w(cb, (V4*)nullptr);
  st4(&dst.q4[d], v);
  dst.px[d] = src.px[s];
  dst.py[d] = src.py[s];
  dst.pz[d] = src.pz[s];
  dst.eps[d] = src.eps[s];
  dst.rho[d] = src.rho[s];
  dst.id[d] = myid;
}

template <class P>
__global__ void k_unload(Consts c, Arrays<P> a, double* io_q, double* io_p, double* io_e) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= c.N) return;
  int64_t k = a.id[t];
  if constexpr (P::mixed) {
    io_q[3 * k] = (double)a.qx[t] * c.scale[0];
    io_q[3 * k + 1] = (double)a.qy[t] * c.scale[1];
    io_q[3 * k + 2] = (double)a.qz[t] * c.scale[2];
  } else {
    io_q[3 * k] = a.qx[t];
    io_q[3 * k + 1] = a.qy[t];
    io_q[3 * k + 2] = a.qz[t];
  }
  io_p[3 * k] = (double)a.px[t];
  io_p[3 * k + 1] = (double)a.py[t];
  io_p[3 * k + 2] = (double)a.pz[t];
  io_e[k] = a.eps[t];
}

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <class P>
void launch_load(const Consts& c, const Workspace& w, cudaStream_t s) {
  if (c.N == 0) return;
  Arrays<P> a = view<P>(w, 0);
  k_load<P><<<blocks_for(c.N, 256), 256, 0, s>>>(c, w.io_q, w.io_p, w.io_e, a, (typename P::Q*)w.qdx,
                                                  (typename P::Q*)w.qdy, (typename P::Q*)w.qdz, w.mrank,
                                                  w.key, w.slot, w.cell_count, w.status);
}

template <class P>
void launch_sort(const Consts& c, const Workspace& w, int from, cudaStream_t s) {
  const int ntiles = (c.ncell + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<ntiles, 256, 0, s>>>(c.ncell, w.cell_count, w.tile_sum);
  k_scan_sums<<<1, 1024, 0, s>>>(ntiles, w.tile_sum, w.cell_start + c.ncell);
  k_scan_apply<<<ntiles, 256, 0, s>>>(c.ncell, w.cell_count, w.cell_start, w.tile_sum);
  if (c.N == 0) return;
  Arrays<P> src = view<P>(w, from), dst = view<P>(w, 1 - from);
  // w.tmp holds 2N entries: bucketed old indices, then their ids
  k_scatter<<<blocks_for(c.N, 256), 256, 0, s>>>(c.N, w.key, w.slot, w.cell_start, src.id, w.tmp,
                                                  w.tmp + c.N);
  k_gather<P><<<blocks_for(c.N, 256), 256, 0, s>>>(
      c, w.tmp, w.tmp + c.N, w.key, w.cell_start, w.rcoord, (const typename P::Q*)w.qdx,
      (const typename P::Q*)w.qdy, (const typename P::Q*)w.qdz, src, dst, w.xmin[0], w.xmin[1],
      w.xmin[2], w.qf4);
}

template <class P>
void launch_unload(const Consts& c, const Workspace& w, int cur, cudaStream_t s) {
  if (c.N == 0) return;
  k_unload<P><<<blocks_for(c.N, 256), 256, 0, s>>>(c, view<P>(w, cur), w.io_q, w.io_p, w.io_e);
}

template void launch_load<Fp64>(const Consts&, const Workspace&, cudaStream_t);
template void launch_load<Mixed>(const Consts&, const Workspace&, cudaStream_t);
template void launch_sort<Fp64>(const Consts&, const Workspace&, int, cudaStream_t);
template void launch_sort<Mixed>(const Consts&, const Workspace&, int, cudaStream_t);
template void launch_unload<Fp64>(const Consts&, const Workspace&, int, cudaStream_t);
template void launch_unload<Mixed>(const Consts&, const Workspace&, int, cudaStream_t);

}  // namespace sdpd
