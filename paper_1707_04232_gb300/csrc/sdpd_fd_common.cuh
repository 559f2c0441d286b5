// sdpd_fd_common.cuh -- block geometry shared by the sweep's schedule
// kernels and its colour kernels: the cells of a 2x2x2 block, local
// coordinates of its particles and owner-cell arithmetic.
#pragma once
#include "sdpd_internal.cuh"

namespace sdpd {

constexpr int kRowWords = kMaxBlock / 32;  // words of one bitmap row

// Cells of the block of owner (ox, oy, oz): start / count in storage order,
// and the local offset of each cell in the block's concatenation.
struct BlockCells {
  int start[8], cnt[8], base[9];
};

__device__ __forceinline__ void block_cells(const Consts& c, int ox, int oy, int oz,
                                            const int32_t* __restrict__ mrank,
                                            const int32_t* __restrict__ cell_start, BlockCells& b) {
  b.base[0] = 0;
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    int cx = ox + (d & 1), cy = oy + ((d >> 1) & 1), cz = oz + ((d >> 2) & 1);
    if (cx >= c.nc[0]) cx -= c.nc[0];
    if (cy >= c.nc[1]) cy -= c.nc[1];
    if (cz >= c.nc[2]) cz -= c.nc[2];
    int r = __ldg(&mrank[cx + c.nc[0] * (cy + c.nc[1] * cz)]);
    b.start[d] = __ldg(&cell_start[r]);
    b.cnt[d] = __ldg(&cell_start[r + 1]) - b.start[d];
    b.base[d + 1] = b.base[d] + b.cnt[d];
  }
}

__device__ __forceinline__ int cell_code_of(const BlockCells& b, int k) {
  int d = 0;
#pragma unroll
  for (int t = 1; t < 8; ++t) d += (k >= b.base[t]);
  return d;
}

// Block-local coordinates of a particle.  Float64: absolute (the minimum
// image is taken per pair, as in the neighbour search).  Mixed: relative to
// the block's lower corner, from the cell-relative coordinates and the exact
// fixed-point distance between cell corners.
template <class P>
struct BlockGeom;

template <>
struct BlockGeom<Fp64> {
  double L[3], halfL[3];
  __device__ void init(const Consts& c, int, int, int, const uint32_t*, const uint32_t*, const uint32_t*) {
    for (int d = 0; d < 3; ++d) { L[d] = c.L[d]; halfL[d] = c.halfL[d]; }
  }
  __device__ __forceinline__ void local(const D4& q, int, double& x, double& y, double& z) const {
    x = q.x; y = q.y; z = q.z;
  }
  __device__ __forceinline__ void disp(double xa, double ya, double za, double xb, double yb, double zb,
                                       double& dx, double& dy, double& dz) const {
    dx = min_image(__dsub_rn(xa, xb), L[0], halfL[0]);
    dy = min_image(__dsub_rn(ya, yb), L[1], halfL[1]);
    dz = min_image(__dsub_rn(za, zb), L[2], halfL[2]);
  }
};

template <>
struct BlockGeom<Mixed> {
  float off[3];  // corner of the upper cell relative to the lower one, per axis
  __device__ void init(const Consts& c, int ox, int oy, int oz, const uint32_t* xmx, const uint32_t* xmy,
                       const uint32_t* xmz) {
    int o[3] = {ox, oy, oz};
    const uint32_t* xm[3] = {xmx, xmy, xmz};
    for (int d = 0; d < 3; ++d) {
      int up = o[d] + 1 >= c.nc[d] ? 0 : o[d] + 1;
      off[d] = (float)(int32_t)(xm[d][up] - xm[d][o[d]]) * (float)c.scale[d];
    }
  }
  __device__ __forceinline__ void local(const F4& q, int code, float& x, float& y, float& z) const {
    x = q.x + ((code & 1) ? off[0] : 0.0f);
    y = q.y + ((code & 2) ? off[1] : 0.0f);
    z = q.z + ((code & 4) ? off[2] : 0.0f);
  }
  __device__ __forceinline__ void disp(float xa, float ya, float za, float xb, float yb, float zb, float& dx,
                                       float& dy, float& dz) const {
    dx = xa - xb; dy = ya - yb; dz = za - zb;
  }
};

__device__ __forceinline__ void owner_coords(const Consts& c, int64_t o, int& ox, int& oy, int& oz) {
  ox = (int)(o % c.nc[0]);
  oy = (int)((o / c.nc[0]) % c.nc[1]);
  oz = (int)(o / ((int64_t)c.nc[0] * c.nc[1]));
}

}  // namespace sdpd
