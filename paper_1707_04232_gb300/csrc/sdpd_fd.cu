// sdpd_fd.cu -- the pairwise fluctuation/dissipation sweep (Sections 3.2-3.3)
// made data-parallel by a conflict-free pair colouring.
//
// Colouring.  A pair whose particles sit in cells a and b (equal or adjacent
// along each axis, since the cell side is >= h) is owned by the cell o that is
// the lower of a and b along each axis (periodically); both cells then lie in
// the 2x2x2 block o + {0,1}^3.  With local cell codes delta in 0..7 (bit k =
// offset along axis k) a pair of cells (dA, dB) of the block is owned by o iff
// dA & dB == 0.  The colour of o is its parity pattern; blocks of one colour
// are disjoint when every cell count is even, so the 8 colours are swept one
// after the other and the blocks of a colour in parallel.
//
// Order inside a block.  Pairs go by (rank(j) - rank(i), rank(i)), rank = the
// position of the id among the block's particles, i the lower id.  Any
// schedule that keeps, for every particle, its pairs in that order gives the
// same result as the sequential sweep; the schedule used here runs the pairs
// in dependency levels (level = length of the longest chain of earlier pairs
// sharing a particle), so the pairs of a level touch disjoint particles.
//
// Three kernels prepare the schedule of every block (it depends on the
// positions only, which are fixed during the sweep): k_sched_enum (one warp
// per block: owned pairs in canonical order), k_sched_walk (one thread per
// block: the dependency level of every pair) and k_sched_bucket (one warp per
// block: pairs bucketed by level); then k_fd_colour runs once per colour (two
// blocks per warp: the pair updates level by level in shared memory).
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

// ---------------------------------------------------------------------------
// Schedule, step 1: owned pairs of every block in canonical order.
// ---------------------------------------------------------------------------
constexpr int kSchedWarps = 2;

struct SchedSmem {
  int32_t id[kMaxBlock];
  uint8_t rank[kMaxBlock];
  uint8_t perm[kMaxBlock];
  uint32_t bits[kRowWords][kMaxBlock];  // bit (lower rank) of row (rank difference); word-major, so
                                        // that lanes reading consecutive rows hit distinct banks
  int32_t rowoff[kMaxBlock + 1];
  int32_t cstart[8], cbase[8], ccnt[8];  // the block's cells: first storage index, offset in the block, count
};

// The owned pairs are read from the neighbour lists of the density pass: a
// particle in block cell dA pairs with owned partners only in the cells
// dB with dA & dB == 0, whose entries sit in known stencil groups of its
// list row.  Each owned pair is met from both of its particles and kept from
// the one with the lower rank.
template <class P>
__global__ void __launch_bounds__(kSchedWarps * 32)
    k_sched_enum(Consts c, Arrays<P> a, const int32_t* __restrict__ cell_start, const int32_t* __restrict__ mrank,
                 const uint32_t* __restrict__ nlist, const uint8_t* __restrict__ nbr_off,
                 uint32_t* __restrict__ hdr, uint16_t* __restrict__ canon, int* status) {
  __shared__ SchedSmem sm_all[kSchedWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t o = (int64_t)blockIdx.x * kSchedWarps + warp;
  if (o >= c.ncell) return;
  SchedSmem& sm = sm_all[warp];
  int ox, oy, oz;
  owner_coords(c, o, ox, oy, oz);
  // the block's 8 cells, one per lane: storage start, count, offset in the
  // block (kept in shared memory, where they are indexed by cell code)
  int ccnt = 0, cst = 0;
  if (lane < 8) {
    int cx = ox + (lane & 1), cy = oy + ((lane >> 1) & 1), cz = oz + ((lane >> 2) & 1);
    if (cx >= c.nc[0]) cx -= c.nc[0];
    if (cy >= c.nc[1]) cy -= c.nc[1];
    if (cz >= c.nc[2]) cz -= c.nc[2];
    const int r = __ldg(&mrank[cx + c.nc[0] * (cy + c.nc[1] * cz)]);
    cst = __ldg(&cell_start[r]);
    ccnt = __ldg(&cell_start[r + 1]) - cst;
  }
  int cinc = ccnt;
#pragma unroll
  for (int sh = 1; sh < 8; sh <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, cinc, sh);
    if (lane >= sh) cinc += t;
  }
  const int nb = __shfl_sync(0xffffffffu, cinc, 7);
  int maxcnt = ccnt;
#pragma unroll
  for (int sh = 4; sh > 0; sh >>= 1) maxcnt = max(maxcnt, __shfl_xor_sync(0xffffffffu, maxcnt, sh));
  maxcnt = __shfl_sync(0xffffffffu, maxcnt, 0);
  if (nb > kMaxBlock) {
    if (lane == 0) { atomicOr(status, kStCapacity); hdr[o] = 0; }
    return;
  }
  if (lane < 8) {
    sm.cstart[lane] = cst;
    sm.cbase[lane] = cinc - ccnt;
    sm.ccnt[lane] = ccnt;
  }
  const int nw = (nb + 31) >> 5;  // bitmap words in use per row
  for (int w = 0; w < nw; ++w)
    for (int row = lane; row < nb; row += 32) sm.bits[w][row] = 0u;
  __syncwarp();
  auto code_of = [&](int k) {
    int d = 0;
#pragma unroll
    for (int t = 1; t < 8; ++t) d += (k >= sm.cbase[t]);
    return d;
  };
  for (int k = lane; k < nb; k += 32) {
    const int d = code_of(k);
    sm.id[k] = a.id[sm.cstart[d] + (k - sm.cbase[d])];
  }
  __syncwarp();
  // rank of each id among the block's ids: every cell's ids are ascending
  int steps = 0;
  while ((1 << steps) <= maxcnt) ++steps;
  for (int k = lane; k < nb; k += 32) {
    const int32_t myid = sm.id[k];
    // per cell: number of ids below myid (branch-free lower bound with a
    // fixed number of halvings, the 8 searches independent of each other)
    int pos[8], len[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) { pos[d] = sm.cbase[d]; len[d] = sm.ccnt[d]; }
    for (int it = 0; it < steps; ++it) {
#pragma unroll
      for (int d = 0; d < 8; ++d) {
        const int half = len[d] >> 1;
        const bool below = len[d] > 0 && sm.id[pos[d] + half] < myid;
        pos[d] = below ? pos[d] + half + 1 : pos[d];
        len[d] = below ? len[d] - half - 1 : half;
      }
    }
    int r = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) r += pos[d] - sm.cbase[d];
    sm.rank[k] = (uint8_t)r;
    sm.perm[r] = (uint8_t)k;
  }
  __syncwarp();
  // Owned entries, spread over the warp: for a chunk of 32 particles (one per
  // lane) and the s-th partner cell of each, a warp prefix sum of the entry
  // counts maps the chunk's entries to lanes, so that the lanes load
  // consecutive entries of a row together and share the work evenly (an
  // owner-cell particle has up to ~80 owned entries, a far-corner one ~3).
  for (int k0 = 0; k0 < nb; k0 += 32) {
    const int k = k0 + lane;
    const bool live = k < nb;
    int dA = 0, g = 0, rk = 0;
    if (live) {
      dA = code_of(k);
      g = sm.cstart[dA] + (k - sm.cbase[dA]);
      rk = sm.rank[k];
    }
    const uint8_t* off = nbr_off + (int64_t)g * 28;
    const int free = 7 & ~dA;
    int dB = free;
    bool more = live;
    for (int sgi = 0; sgi < 8; ++sgi) {  // partner cells dB: subsets of the complement of dA
      int e0 = 0, n = 0, myB = 0;
      if (more) {
        const int sx = ((dB & 1) - (dA & 1)) + 1, sy = (((dB >> 1) & 1) - ((dA >> 1) & 1)) + 1,
                  sz = (((dB >> 2) & 1) - ((dA >> 2) & 1)) + 1;
        const int st = sx + 3 * sy + 9 * sz;
        e0 = off[st];
        n = off[st + 1] - e0;
        myB = dB;
        if (dB == 0) more = false;
        else dB = (dB - 1) & free;
      }
      int incl = n;
#pragma unroll
      for (int sh = 1; sh < 32; sh <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, sh);
        if (lane >= sh) incl += t;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      if (total == 0) {
        if (!__any_sync(0xffffffffu, more)) break;
        continue;
      }
      const int excl = incl - n;
      const int packed = (myB << 8) | e0;  // partner cell and first entry of this lane's segment
      // kDeep rounds of 32 entries per iteration, all list loads issued
      // before any is used
      constexpr int kDeep = 4;
      for (int t0 = 0; t0 < total; t0 += 32 * kDeep) {
        int o_pk[kDeep], o_rk[kDeep], o_q[kDeep];
        uint32_t ent[kDeep];
#pragma unroll
        for (int h = 0; h < kDeep; ++h) {
          const int t = t0 + 32 * h + lane;
          // owner lane: the number of lanes whose inclusive count is <= t
          int pos = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(0xffffffffu, incl, pos + step - 1);
            if (v <= t) pos += step;
          }
          const int src = min(pos, 31);
          o_pk[h] = __shfl_sync(0xffffffffu, packed, src);
          const int o_ex = __shfl_sync(0xffffffffu, excl, src);
          const int o_g = __shfl_sync(0xffffffffu, g, src);
          o_rk[h] = __shfl_sync(0xffffffffu, rk, src);
          o_q[h] = t < total ? (o_pk[h] & 255) + (t - o_ex) : -1;
          ent[h] = o_q[h] >= 0 ? __ldg(&nlist[(int64_t)o_g * c.nbr_cap + o_q[h]]) : 0u;
        }
#pragma unroll
        for (int h = 0; h < kDeep; ++h) {
          if (o_q[h] >= 0) {
            const int oB = o_pk[h] >> 8;
            const int j = (int)(ent[h] >> 6);
            const int rj = sm.rank[sm.cbase[oB] + (j - sm.cstart[oB])];
            if (o_rk[h] < rj) atomicOr(&sm.bits[o_rk[h] >> 5][rj - o_rk[h]], 1u << (o_rk[h] & 31));
          }
        }
      }
      if (!__any_sync(0xffffffffu, more)) break;
    }
  }
  __syncwarp();
  // exclusive scan of the row populations, 32 consecutive rows at a time
  int npairs = 0;
  for (int r0 = 0; r0 < nb; r0 += 32) {
    const int rr = r0 + lane;
    int n = 0;
    if (rr >= 1 && rr < nb)
      for (int w = 0; w < nw; ++w) n += __popc(sm.bits[w][rr]);
    int incl = n;
#pragma unroll
    for (int sh = 1; sh < 32; sh <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, sh);
      if (lane >= sh) incl += t;
    }
    sm.rowoff[rr] = npairs + incl - n;
    npairs += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (npairs > kMaxPairs) {
    if (lane == 0) { atomicOr(status, kStCapacity); hdr[o] = 0; }
    return;
  }
  __syncwarp();
  // write the pairs row by row (difference ascending), lower rank ascending
  uint16_t* out = canon + o * kMaxPairs;
  for (int rr = 1 + lane; rr < nb; rr += 32) {
    int pos = sm.rowoff[rr];
    for (int w = 0; w < nw; ++w) {
      uint32_t bits = sm.bits[w][rr];
      while (bits) {
        const int bit = __ffs(bits) - 1;
        bits &= bits - 1;
        const int lo = w * 32 + bit;
        out[pos++] = (uint16_t)(sm.perm[lo] | (sm.perm[lo + rr] << 8));
      }
    }
  }
  if (lane == 0) hdr[o] = (uint32_t)npairs;
}

// Levels, step 1: one thread per block walks that block's canonical list and
// records the level of every pair (the longest chain of earlier pairs sharing
// a particle).  A warp handles 32 consecutive blocks and moves their lists
// and levels through shared memory 32 entries at a time, so every global
// access is coalesced.
constexpr int kLevelThreads = 32;
constexpr int kTile = 32;

__global__ void __launch_bounds__(kLevelThreads) k_sched_walk(int64_t ncell, uint32_t* __restrict__ hdr,
                                                            const uint16_t* __restrict__ canon,
                                                            uint8_t* __restrict__ level_of, int* status) {
  __shared__ uint8_t last_s[kMaxBlock][kLevelThreads];  // level after which a particle is free
  __shared__ uint16_t tile[kLevelThreads][kTile + 1];
  __shared__ uint8_t ltile[kLevelThreads][kTile + 4];
  const int t = threadIdx.x;
  const int64_t o0 = (int64_t)blockIdx.x * kLevelThreads;
  const int64_t o = o0 + t;
  const bool live = o < ncell;
  const int np = live ? (int)(hdr[o] & 0xffffu) : 0;
  int npmax = np;
  for (int s = 16; s > 0; s >>= 1) npmax = max(npmax, __shfl_xor_sync(0xffffffffu, npmax, s));
  for (int k = 0; k < kMaxBlock; ++k) last_s[k][t] = 0;
  int nlev = 0;
  bool overflow = false;
  for (int k0 = 0; k0 < npmax; k0 += kTile) {
    __syncwarp();
    for (int j = 0; j < kLevelThreads; ++j) {
      const int64_t oj = o0 + j;
      if (oj < ncell) tile[j][t] = canon[oj * kMaxPairs + k0 + t];
    }
    __syncwarp();
    const int kn = min(kTile, np - k0);
    for (int k = 0; k < kn; ++k) {
      const uint16_t pr = tile[t][k];
      const int u = pr & 255, v = pr >> 8;
      const int L = max(last_s[u][t], last_s[v][t]);
      if (L >= kMaxLevels) { overflow = true; ltile[t][k] = 0; continue; }
      last_s[u][t] = last_s[v][t] = (uint8_t)(L + 1);
      ltile[t][k] = (uint8_t)L;
      nlev = max(nlev, L + 1);
    }
    __syncwarp();
    for (int j = 0; j < kLevelThreads; ++j) {
      const int64_t oj = o0 + j;
      if (oj < ncell) level_of[oj * kMaxPairs + k0 + t] = ltile[j][t];
    }
  }
  if (live) {
    if (overflow) {
      atomicOr(status, kStCapacity);
      hdr[o] = 0;
    } else {
      hdr[o] = (uint32_t)np | ((uint32_t)nlev << 16);
    }
  }
}

// Levels, step 2: one warp per block buckets the canonical list by level
// (order inside a level is free: its pairs touch disjoint particles) and
// writes the level offsets.
constexpr int kBucketWarps = 4;

__global__ void __launch_bounds__(kBucketWarps * 32) k_sched_bucket(int64_t ncell, const uint32_t* __restrict__ hdr,
                                                                  const uint16_t* __restrict__ canon,
                                                                  const uint8_t* __restrict__ level_of,
                                                                  uint16_t* __restrict__ lvl,
                                                                  uint16_t* __restrict__ pairs) {
  __shared__ int32_t cnt_s[kBucketWarps][kMaxLevels + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t o = (int64_t)blockIdx.x * kBucketWarps + warp;
  if (o >= ncell) return;
  const uint32_t hd = hdr[o];
  const int np = (int)(hd & 0xffffu), nlev = (int)(hd >> 16);
  int32_t* cnt = cnt_s[warp];
  for (int L = lane; L <= kMaxLevels; L += 32) cnt[L] = 0;
  __syncwarp();
  const uint16_t* in = canon + o * kMaxPairs;
  const uint8_t* lv = level_of + o * kMaxPairs;
  for (int k = lane; k < np; k += 32) atomicAdd(&cnt[lv[k]], 1);
  __syncwarp();
  // exclusive scan over nlev (<= 255) levels: 8 per lane
  int v[8], sum = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int L = lane * 8 + q;
    v[q] = L < nlev ? cnt[L] : 0;
    sum += v[q];
  }
  int incl = sum;
  for (int s = 1; s < 32; s <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, s);
    if (lane >= s) incl += t;
  }
  int run = incl - sum;
  uint16_t* off = lvl + o * (kMaxLevels + 1);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int L = lane * 8 + q;
    if (L < nlev) {
      off[L] = (uint16_t)run;
      cnt[L] = run;
    }
    run += v[q];
  }
  if (lane == 31) off[nlev] = (uint16_t)run;
  __syncwarp();
  uint16_t* out = pairs + o * kMaxPairs;
  for (int k = lane; k < np; k += 32) out[atomicAdd(&cnt[lv[k]], 1)] = in[k];
}

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
__device__ __forceinline__ double rsqrt(double x) { return 1.0 / ::sqrt(x); }
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

// Box-Muller normals and the uniform of one pair at one sweep (see
// pair_randoms); the float32 path uses the hardware log and sin/cos.
__device__ __forceinline__ void pair_randoms_fast(uint64_t seed, uint64_t sweep, uint64_t idi, uint64_t idj,
                                                  float G[3], float* U) {
  uint64_t w[4];
  philox4x64_10(sweep, idi, idj, 0ull, seed, 0ull, w);
  const float two23 = 1.0f / 8388608.0f, twopi = 6.28318530717958647692f;
  const float u0 = ((float)(uint32_t)(w[0] >> 41) + 0.5f) * two23;
  const float u1 = ((float)(uint32_t)(w[1] >> 41) + 0.5f) * two23;
  const float R = fm::sqrt(-2.0f * __logf(u0));
  float sn, cs;
  __sincosf(twopi * u1, &sn, &cs);
  G[0] = R * cs;
  G[1] = R * sn;
  const float u2 = ((float)(uint32_t)(w[2] >> 41) + 0.5f) * two23;
  const float u3 = ((float)((uint32_t)(w[2] & 0xffffffffull) >> 9) + 0.5f) * two23;
  G[2] = fm::sqrt(-2.0f * __logf(u2)) * __cosf(twopi * u3);
  *U = ((float)(uint32_t)(w[3] >> 41) + 0.5f) * two23;
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
template <class R>
__device__ __forceinline__ void pair_coeffs(const FDConst<R>& k, R kpar, R kperp, R ei, R ej, R& apar,
                                            R& aperp, R& zpar, R& zperp, R& xpar, R& xperp) {
  const R Ti = ei * k.inv_C_K, Tj = ej * k.inv_C_K;
  const R sT = Ti + Tj;
  const R hT = fm::div(Ti * Tj, sT);
  const R omd = R(1) - fm::div(k.kB * hT * k.two_over_CK, sT);
  xpar = R(-2) * kpar * omd * k.dt_over_m;  // log alpha per direction
  xperp = R(-2) * kperp * omd * k.dt_over_m;
  apar = fm::exp(xpar);
  aperp = fm::exp(xperp);
  const R s = fm::div(k.four_kB_over_m * hT, omd);
  zpar = fm::sqrt(s * -fm::expm1(R(2) * xpar));
  zperp = fm::sqrt(s * -fm::expm1(R(2) * xperp));
}

// State-dependent part of one pair update on (p_i, p_j) with internal
// energies (ei, ej) in the arithmetic type R, given the pair's unit vector
// e = r_ij / r_ij, base = F(r_ij) / (rho_i rho_j) and its random numbers.
// Returns 0 accept, 1 energy-bound reject, 2 Metropolis reject; deps receives
// the energy change shared by the two particles (applied by the caller on
// acceptance).  exact_bound: float64 re-check of the energy bound for the
// mixed path when its float32 margin is not decisive; it returns the smaller
// new internal energy in float64.
template <class P, class ExactBound>
__device__ __forceinline__ int fd_pair(const FDConst<typename P::R>& k, typename P::R ex, typename P::R ey,
                                       typename P::R ez, typename P::R base, const typename P::R G[3],
                                       typename P::R U, typename P::R* pi, typename P::R* pj,
                                       typename P::R ei, typename P::R ej, typename P::R& deps,
                                       typename P::R& margin, bool& negative, ExactBound exact_bound) {
  using R = typename P::R;
  const R kpar = k.kpar_m2 * base, kperp = k.kperp_m2 * base;
  margin = R(0);
  deps = R(0);
  if (!(kperp > R(0)) || !(kpar > R(0))) return 0;  // at r = h the pair does nothing
  const R vx = (pi[0] - pj[0]) * k.inv_m, vy = (pi[1] - pj[1]) * k.inv_m, vz = (pi[2] - pj[2]) * k.inv_m;
  R apar, aperp, zpar, zperp;
  R xfpar, xfperp;
  pair_coeffs(k, kpar, kperp, ei, ej, apar, aperp, zpar, zperp, xfpar, xfperp);
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
  if constexpr (P::mixed) {
    // -1/2 of the kinetic-energy change of the stored momenta, as a sum of
    // (new - old)(new + old) products so float32 carries no cancellation
    const float dk = (nix - pi[0]) * (nix + pi[0]) + (niy - pi[1]) * (niy + pi[1]) +
                     (niz - pi[2]) * (niz + pi[2]) + (njx - pj[0]) * (njx + pj[0]) +
                     (njy - pj[1]) * (njy + pj[1]) + (njz - pj[2]) * (njz + pj[2]);
    deps = -0.25f * k.inv_m * dk;
  } else {
    const double ko = pi[0] * pi[0] + pj[0] * pj[0] + pi[1] * pi[1] + pj[1] * pj[1] + pi[2] * pi[2] +
                      pj[2] * pj[2];
    const double kn = nix * nix + njx * njx + niy * niy + njy * njy + niz * niz + njz * njz;
    deps = -0.5 * (kn - ko) * (0.5 * k.inv_m);
  }
  // energy bound, Eq. (energy-bound): both new internal energies > 0
  const R emin_old = ei < ej ? ei : ej;
  R emin = emin_old + deps;
  if constexpr (P::mixed) {
    // float32 decides unless the margin is within a few ulps of zero
    if (fabsf(emin) <= 8.0f * 1.1920929e-7f * emin_old) emin = exact_bound(deps) > 0.0 ? 1.0f : -1.0f;
  }
  margin = emin;
  int decision = 0;
  if (k.scheme == SDPD_SCHEME_SSA) {
    if (!(emin > R(0))) negative = true;
  } else if (!(emin > R(0))) {
    decision = 1;
  } else if (k.scheme == SDPD_SCHEME_EMS) {
    // Metropolis ratio, Eq. (metropolis-ratio): the reverse move from v'
    // with the coefficients at the proposed energies
    R bpar, bperp, ypar, yperp, xrpar, xrperp;
    pair_coeffs(k, kpar, kperp, ei + deps, ej + deps, bpar, bperp, ypar, yperp, xrpar, xrperp);
    R quad;
    if constexpr (P::mixed) {
      // reverse noise of the proposal v' = A v + B G:
      // B'^-1 (v - A' v') = B'^-1 [(I - A' A) v - A' B G], each direction
      // scaled separately, I - A' A from expm1 of the summed exponents; in
      // float32 the literal v - A' v' loses its digits to cancellation when
      // zt -> 0 (pairs near the cut-off)
      const R cpar_r = -fm::expm1(xfpar + xrpar), cperp_r = -fm::expm1(xfperp + xrperp);
      const R qpar = fm::div(cpar_r * vpar - bpar * zpar * gpar, ypar);
      const R ip = fm::div(R(1), yperp);
      const R qx = (cperp_r * (vx - vpar * ex) - bperp * zperp * (G[0] - gpar * ex)) * ip;
      const R qy = (cperp_r * (vy - vpar * ey) - bperp * zperp * (G[1] - gpar * ey)) * ip;
      const R qz = (cperp_r * (vz - vpar * ez) - bperp * zperp * (G[2] - gpar * ez)) * ip;
      quad = qpar * qpar + qx * qx + qy * qy + qz * qz;
    } else {
      // reverse noise B'^-1 (v - A' v') from the proposed v' itself
      const R wpar = ex * wx + ey * wy + ez * wz;
      const R cb = (bpar - bperp) * wpar;
      const R bx = vx - (bperp * wx + cb * ex), by = vy - (bperp * wy + cb * ey), bz = vz - (bperp * wz + cb * ez);
      const R spar = ex * bx + ey * by + ez * bz;
      const R ip = fm::div(R(1), yperp);
      const R cq = (fm::div(R(1), ypar) - ip) * spar;
      const R qx = bx * ip + cq * ex, qy = by * ip + cq * ey, qz = bz * ip + cq * ez;
      quad = qx * qx + qy * qy + qz * qz;
    }
    const R g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    // log|B(v)| - log|B(v')| with |B| = zt_par zt_perp^2
    const R ldet = fm::log(fm::div(zpar * zperp * zperp, ypar * yperp * yperp));
    // (S(eps') - S(eps))/kB - (log T(eps') - log T(eps)) = (C_K/kB - 1) log(eps'/eps)
    // summed over the two particles: log1p(x) + log1p(y) = log1p(x + y + x y)
    const R xi = fm::div(deps, ei), xj = fm::div(deps, ej);
    const R ent = k.CKm1 * fm::log1p(xi + xj + xi * xj);
    const R a = R(0.5) * (g2 - quad) + ldet + ent;
    const R mg = a - fm::log(U);
    margin = mg;
    if (mg < R(0)) decision = 2;  // U > exp(a)
  }
  if (decision == 0) {
    pi[0] = nix; pi[1] = niy; pi[2] = niz;
    pj[0] = njx; pj[1] = njy; pj[2] = njz;
  }
  return decision;
}

// ---------------------------------------------------------------------------
// One colour of the sweep.  A warp runs kOwnersPerWarp blocks of the colour
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
constexpr int kOwnersPerWarp = 2;
constexpr int kGroupLanes = 32 / kOwnersPerWarp;
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
struct FdSmem {
  R px[kMaxBlock], py[kMaxBlock], pz[kMaxBlock];
  R e[kMaxBlock];    // energy at hand (float64 path: the energy itself)
  R acc[kMaxBlock];  // mixed path: float32 sum of this visit's energy changes
  int32_t cst[8], cbs[8];  // the block's cells: first storage index, offset in the block
  // staged pair data of the current chunk
  R G0[kChunk], G1[kChunk], G2[kChunk], U[kChunk];
  R ex[kChunk], ey[kChunk], ez[kChunk], base[kChunk];
  uint16_t pr[kChunk];
  uint16_t off[kMaxLevels + 1];  // level offsets of the block's pair list
};

template <class P>
constexpr int fd_warps() { return P::mixed ? 2 : 1; }

template <class P, int KIND>
__global__ void __launch_bounds__(fd_warps<P>() * 32, P::mixed ? 8 : 4)
    k_fd_colour(Consts c, FDConst<typename P::R> k, Arrays<P> a, typename P::V4* __restrict__ qp4,
                const int32_t* __restrict__ cell_start, const int32_t* __restrict__ mrank,
                const uint32_t* __restrict__ xmx, const uint32_t* __restrict__ xmy,
                const uint32_t* __restrict__ xmz, const uint32_t* __restrict__ hdr,
                const uint16_t* __restrict__ lvl, const uint16_t* __restrict__ pairs, int colour, uint64_t seed,
                const unsigned long long* __restrict__ sweep_ptr, unsigned long long* counters, int* status,
                sdpd_pair_rec* recs, unsigned long long* rec_count, int64_t rec_cap) {
  using R = typename P::R;
  constexpr int W = fd_warps<P>();
  __shared__ FdSmem<R> sm_all[W][kOwnersPerWarp];
  const uint64_t sweep = *sweep_ptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / kGroupLanes, gl = lane % kGroupLanes;
  const int hx = c.nc[0] >> 1, hy = c.nc[1] >> 1, hz = c.nc[2] >> 1;
  const int64_t nown = (int64_t)hx * hy * hz;
  const int64_t w = ((int64_t)blockIdx.x * W + warp) * kOwnersPerWarp + grp;
  FdSmem<R>& sm = sm_all[warp][grp];
  int np = 0, nlev = 0;
  int64_t o = 0;
  int ox = 0, oy = 0, oz = 0;
  if (w < nown) {
    ox = 2 * (int)(w % hx) + (colour & 1);
    oy = 2 * (int)((w / hx) % hy) + ((colour >> 1) & 1);
    oz = 2 * (int)(w / ((int64_t)hx * hy)) + ((colour >> 2) & 1);
    o = ox + (int64_t)c.nc[0] * (oy + (int64_t)c.nc[1] * oz);
    const uint32_t hd = hdr[o];
    np = (int)(hd & 0xffffu);
    nlev = (int)(hd >> 16);
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
  for (int q = gl; q < nb; q += kGroupLanes) {
    const int g = gidx(q);
    sm.px[q] = a.px[g]; sm.py[q] = a.py[g]; sm.pz[q] = a.pz[g];
    sm.e[q] = (R)a.eps[g];
    sm.acc[q] = R(0);
  }
  for (int L = gl; L <= nlev; L += kGroupLanes) sm.off[L] = lvl[o * (kMaxLevels + 1) + L];
  __syncwarp();
  const uint16_t* off = sm.off;
  const uint16_t* pl = pairs + o * kMaxPairs;
  const R inv_h = k.inv_h, cF = k.cF;
  unsigned long long n_acc = 0, n_rb = 0, n_rm = 0, n_tot = 0;
  bool negative = false, bad = false;
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
      const int ga = gidx(ia), gb = gidx(ib);
      R xa, ya, za, xb, yb, zb, rx, ry, rz;
      const typename P::V4 qa = ld4(&a.q4[ga]), qb = ld4(&a.q4[gb]);
      geo.local(qa, block_code(qa.w, ox, oy, oz), xa, ya, za);
      geo.local(qb, block_code(qb.w, ox, oy, oz), xb, yb, zb);
      geo.disp(xa, ya, za, xb, yb, zb, rx, ry, rz);
      const R r2 = r2_of(rx, ry, rz);
      const R inv_r = fm::rsqrt(r2);
      const int slot = t - cbeg;
      sm.pr[slot] = pr;
      sm.ex[slot] = rx * inv_r;
      sm.ey[slot] = ry * inv_r;
      sm.ez[slot] = rz * inv_r;
      sm.base[slot] = fm::div(kernel_F<KIND>(r2 * inv_r * inv_h, cF), a.rho[ga] * a.rho[gb]);
      R G[3], U;
      pair_randoms_fast(seed, sweep, (uint64_t)a.id[ga], (uint64_t)a.id[gb], G, &U);
      sm.G0[slot] = G[0]; sm.G1[slot] = G[1]; sm.G2[slot] = G[2]; sm.U[slot] = U;
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
        const R ea = sm.e[ia], eb = sm.e[ib];
        const R G[3] = {sm.G0[slot], sm.G1[slot], sm.G2[slot]};
        R deps, margin;
        // float64 bound for the mixed path: energies at load plus this visit's sums
        auto exact = [&](R dv) -> double {
          const double da = a.eps[gidx(ia)] + (double)sm.acc[ia];
          const double db = a.eps[gidx(ib)] + (double)sm.acc[ib];
          return fmin(da, db) + (double)dv;
        };
        const int dcs = fd_pair<P>(k, sm.ex[slot], sm.ey[slot], sm.ez[slot], sm.base[slot], G, sm.U[slot], pa,
                                   pb, ea, eb, deps, margin, negative, exact);
        if (dcs == 0) {
          sm.px[ia] = pa[0]; sm.py[ia] = pa[1]; sm.pz[ia] = pa[2];
          sm.px[ib] = pb[0]; sm.py[ib] = pb[1]; sm.pz[ib] = pb[2];
          sm.e[ia] = ea + deps;
          sm.e[ib] = eb + deps;
          if constexpr (P::mixed) {
            sm.acc[ia] += deps;
            sm.acc[ib] += deps;
          }
          bad |= !isfinite(sm.e[ia]) || !isfinite(sm.e[ib]);
        }
        ++n_tot;
        n_acc += dcs == 0;
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
            rc.margin = (double)margin;
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
  const R pi_coef = (R)(c.c_rho / (c.C_K * c.m));
  for (int q = gl; q < nb; q += kGroupLanes) {
    const int g = gidx(q);
    a.px[g] = sm.px[q]; a.py[g] = sm.py[q]; a.pz[g] = sm.pz[q];
    double e;
    if constexpr (P::mixed) e = a.eps[g] + (double)sm.acc[q];  // one float64 update per visit
    else e = sm.e[q];
    a.eps[g] = e;
    // pressure over rho^2 of the new energy, Eq. (pg-eos): pi = c_rho eps / (C_K m rho)
    qp4[g].w = (R)e * pi_coef / a.rho[g];
  }
  // counters
  for (int s = 16; s > 0; s >>= 1) {
    n_tot += __shfl_xor_sync(0xffffffffu, n_tot, s);
    n_acc += __shfl_xor_sync(0xffffffffu, n_acc, s);
    n_rb += __shfl_xor_sync(0xffffffffu, n_rb, s);
    n_rm += __shfl_xor_sync(0xffffffffu, n_rm, s);
  }
  const unsigned any_neg = __any_sync(0xffffffffu, negative), any_bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    if (n_tot) {
      atomicAdd(&counters[0], n_tot);
      atomicAdd(&counters[1], n_acc);
      atomicAdd(&counters[2], n_rb);
      atomicAdd(&counters[3], n_rm);
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
  k.scheme = c.scheme;
  return k;
}

template <class P>
void launch_fd_schedule(const Consts& c, const Workspace& w, int cur, cudaStream_t s) {
  if (c.N == 0) return;
  Arrays<P> a = view<P>(w, cur);
  uint16_t* canon = w.sched_pair + (size_t)c.ncell * kMaxPairs;
  const unsigned gs = (unsigned)((c.ncell + kSchedWarps - 1) / kSchedWarps);
  k_sched_enum<P><<<gs, kSchedWarps * 32, 0, s>>>(c, a, w.cell_start, w.mrank, w.nlist, w.nbr_off,
                                                   w.sched_hdr, canon, w.status);
  k_sched_walk<<<(unsigned)((c.ncell + kLevelThreads - 1) / kLevelThreads), kLevelThreads, 0, s>>>(
      c.ncell, w.sched_hdr, canon, w.level_of, w.status);
  k_sched_bucket<<<(unsigned)((c.ncell + kBucketWarps - 1) / kBucketWarps), kBucketWarps * 32, 0, s>>>(
      c.ncell, w.sched_hdr, canon, w.level_of, w.sched_lvl, w.sched_pair);
}

__global__ void k_sweep_set(unsigned long long* sweep, unsigned long long v) { *sweep = v; }
__global__ void k_sweep_advance(unsigned long long* sweep) { *sweep += 1ull; }

void launch_set_sweep(const Workspace& w, unsigned long long value, cudaStream_t s) {
  k_sweep_set<<<1, 1, 0, s>>>(w.sweep, value);
}
void launch_advance_sweep(const Workspace& w, cudaStream_t s) { k_sweep_advance<<<1, 1, 0, s>>>(w.sweep); }

template <class P>
void launch_fd_colours(const Consts& c, const Workspace& w, int cur, double dt, uint64_t seed, int record,
                       cudaStream_t s) {
  if (c.N == 0) return;
  using R = typename P::R;
  Arrays<P> a = view<P>(w, cur);
  const FDConst<R> k = fd_const<R>(c, dt);
  constexpr int W = fd_warps<P>();
  const int64_t nown = (int64_t)(c.nc[0] / 2) * (c.nc[1] / 2) * (c.nc[2] / 2);
  const int64_t per_block = (int64_t)W * kOwnersPerWarp;
  const unsigned gf = (unsigned)((nown + per_block - 1) / per_block);
  auto qp4 = (typename P::V4*)w.qp4;
  sdpd_pair_rec* recs = record ? w.pair_recs : nullptr;
  for (int col = 0; col < 8; ++col) {
    if (c.kernel == SDPD_KERNEL_LUCY)
      k_fd_colour<P, SDPD_KERNEL_LUCY><<<gf, W * 32, 0, s>>>(
          c, k, a, qp4, w.cell_start, w.mrank, w.xmin[0], w.xmin[1], w.xmin[2], w.sched_hdr, w.sched_lvl,
          w.sched_pair, col, seed, w.sweep, w.counters, w.status, recs, w.pair_rec_count, w.pair_rec_cap);
    else
      k_fd_colour<P, SDPD_KERNEL_CUBIC><<<gf, W * 32, 0, s>>>(
          c, k, a, qp4, w.cell_start, w.mrank, w.xmin[0], w.xmin[1], w.xmin[2], w.sched_hdr, w.sched_lvl,
          w.sched_pair, col, seed, w.sweep, w.counters, w.status, recs, w.pair_rec_count, w.pair_rec_cap);
  }
}

template void launch_fd_schedule<Fp64>(const Consts&, const Workspace&, int, cudaStream_t);
template void launch_fd_schedule<Mixed>(const Consts&, const Workspace&, int, cudaStream_t);
template void launch_fd_colours<Fp64>(const Consts&, const Workspace&, int, double, uint64_t, int, cudaStream_t);
template void launch_fd_colours<Mixed>(const Consts&, const Workspace&, int, double, uint64_t, int, cudaStream_t);

}  // namespace sdpd
