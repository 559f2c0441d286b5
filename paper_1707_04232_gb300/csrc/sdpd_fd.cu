// sdpd_fd.cu -- the pairwise fluctuation/dissipation sweep (Sections 3.2-3.3)
// made data-parallel by a conflict-free pair colouring.
//
// Colouring.  A pair whose particles sit in cells a and b (equal or adjacent
// along each axis, since the cell side is >= h) is owned by a cell o such that
// both cells lie in the 2x2x2 block o + {0,1}^3: along an axis where a and b
// are adjacent o takes the lower of the two (periodically); along an axis
// where they coincide either block holding the coordinate would do, and bit
// k of owner_bits(lower id) picks the one where the shared cell is the lower
// (0) or upper (1) cell of the block.  With local cell codes dA, dB in 0..7
// (bit k = offset along axis k, A the lower id) the block owns the pair iff
// dA and dB agree with the owner bits wherever they coincide.  Spreading a
// particle's pairs over the colours this way roughly halves the longest
// chain of pairs in a block compared with always taking the lower block.
// The colour of o is its parity pattern; blocks of one colour are disjoint
// when every cell count is even, so the 8 colours are swept one after the
// other and the blocks of a colour in parallel.
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
// block: pairs bucketed by level); two more order each colour's blocks by
// depth (k_sched_order_scan, k_sched_order_scatter); then k_fd_colour (sdpd_fd_colour.cuh)
// runs once per colour: the pair updates level by level in shared memory,
// one or two blocks per warp as the launch's block schedule says.
#include "sdpd_fd_common.cuh"

namespace sdpd {


// ---------------------------------------------------------------------------
// Schedule, step 1: owned pairs of every block in canonical order, found
// from the positions of the block's particles.  One thread block of
// kEnumThreads threads per owner cell stages the particles of the block's 8
// cells in shared memory (ids, coordinates) and tests every candidate pair
// with the neighbour predicate r^2 < h^2 of the pair passes:
//   * float64: absolute coordinates and the minimum image, after the float32
//     pre-test of the density pass (which skips only pairs with r >= h);
//   * mixed: block-local float32 coordinates, the arithmetic the colour
//     kernel uses for the pair's geometry.
// Ranks.  Every cell holds its particles by ascending id, so the rank of a
// particle among the block's ids is the sum over the 8 cells of the number
// of smaller ids there (lb[k][d'] = ids in cell d' below particle k's, by
// binary search; in its own cell, its position).
// Candidates.  A particle A (as the lower id of a pair) in block cell dA has
// owned partners only in the cells dB that agree with dA where dA agrees
// with A's owner bits and differ from dA elsewhere, and only among the ids
// above its own: the suffix of cell dB from lb[A][dB] on (from A + 1 in its
// own cell).  One thread walks each particle's candidates, the particles
// taken in order of their number of candidates (a counting sort).
// Found pairs set bit rank(i) of row d = rank(j) - rank(i) of a triangular
// bitmap (row d holds nb - d bits in whole words: it starts at word
// F(nb - 1) - F(nb - d) with F(n) = sum_{k <= n} ceil(k / 32)), which is then
// read out row by row.  The kernel is kept small (about 13 KB of shared
// memory for the mixed path) so that 16 blocks share an SM: its phases are
// short and wait on memory, and other blocks fill the gaps.
// ---------------------------------------------------------------------------
constexpr int kEnumThreads = 128;
constexpr int kTriWords = 1152;  // >= F(255) = 1144: a triangle of 256 rows

// words of the first rows of the triangular bitmap: F(n) = sum_{k=1..n} ceil(k/32)
__device__ __forceinline__ int tri_f(int n) {
  const int q = n >> 5, s = n & 31;
  return 16 * q * (q + 1) + s * (q + 1);
}

template <class R>
struct EnumSmem {
  // coordinates: float64 absolute, mixed block-local (w unused)
  typename std::conditional<std::is_same<R, double>::value, D4, float4>::type x[kMaxBlock];
  float4 f[std::is_same<R, double>::value ? kMaxBlock : 1];  // float64: float32 copies for the pre-test
  uint32_t bits[kTriWords];
  int32_t id[kMaxBlock];
  uint8_t lb[kMaxBlock][8];  // ids of each cell below the particle's (own cell: its position)
  uint16_t rowoff[kMaxBlock];
  uint16_t rowbase[kMaxBlock];  // first word of each row of the bitmap
  uint8_t ncand[kMaxBlock];     // each particle's number of candidates (clamped to 255)
  uint8_t order[kMaxBlock];     // the particles by number of candidates, most first
  int32_t hist[kMaxBlock + 1];  // particles by number of candidates (clamped to 255)
  uint8_t code[kMaxBlock];   // block cell of each particle
  uint8_t rank[kMaxBlock];
  uint8_t perm[kMaxBlock];
  int32_t cstart[8], cbase[9];
  int32_t npairs, nb;
};

template <class P>
__global__ void __launch_bounds__(kEnumThreads)
    k_sched_enum(Consts c, Arrays<P> a, const int32_t* __restrict__ cell_start, const int32_t* __restrict__ mrank,
                 const uint32_t* __restrict__ xmx, const uint32_t* __restrict__ xmy,
                 const uint32_t* __restrict__ xmz, const float4* __restrict__ qf4, uint32_t* __restrict__ hdr,
                 uint16_t* __restrict__ canon, uint32_t* __restrict__ blk_hist, uint32_t* __restrict__ big_count) {
  using R = typename P::R;
  __shared__ EnumSmem<R> sm;
  const int t = threadIdx.x, lane = t & 31;
  if (blockIdx.x == 0) {  // the depth histogram and the lists of blocks beyond capacity that k_sched_walk fills
    for (int k = t; k < 8 * 256; k += kEnumThreads) blk_hist[k] = 0u;
    if (t < 16) big_count[t] = 0u;
  }
  const int o = blockIdx.x;  // owner cell (fewer than 2^31 cells)
  const int ox = o % c.nc[0], oy = (o / c.nc[0]) % c.nc[1], oz = o / (c.nc[0] * c.nc[1]);
  // the block's 8 cells: storage start, count and offset in the block
  if (t < 32) {
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
      const int v = __shfl_up_sync(0xffffffffu, cinc, sh);
      if (lane >= sh) cinc += v;
    }
    if (lane < 8) {
      sm.cstart[lane] = cst;
      sm.cbase[lane] = cinc - ccnt;
    }
    if (lane == 7) {
      sm.cbase[8] = cinc;
      sm.nb = cinc;
    }
    if (lane == 0) sm.npairs = 0;
  }
  __syncthreads();
  const int nb = sm.nb;
  if (nb > kMaxBlock) {  // beyond capacity: swept pair by pair (see kHdrBig)
    if (t == 0) hdr[o] = kHdrBig;
    return;
  }
  const int ntri = nb > 1 ? tri_f(nb - 1) : 0;  // words of the bitmap in use
  for (int q = t; q < ntri; q += kEnumThreads) sm.bits[q] = 0u;
  BlockGeom<P> geo;
  geo.init(c, ox, oy, oz, xmx, xmy, xmz);
  int cb[9];
#pragma unroll
  for (int u = 0; u < 9; ++u) cb[u] = sm.cbase[u];
  for (int k = t; k < nb; k += kEnumThreads) {  // the particles
    int d = 0;
#pragma unroll
    for (int u = 1; u < 8; ++u) d += (k >= cb[u]);
    const int g = sm.cstart[d] + (k - sm.cbase[d]);
    sm.id[k] = a.id[g];
    sm.code[k] = (uint8_t)d;
    R x, y, zz;
    geo.local(ld4(&a.q4[g]), d, x, y, zz);
    sm.x[k].x = x; sm.x[k].y = y; sm.x[k].z = zz;
    if constexpr (!P::mixed) sm.f[k] = __ldg(&qf4[g]);
  }
  __syncthreads();
  // lower bounds: for every particle and cell, the ids of the cell below the
  // particle's, by branch-free binary searches of a fixed length, the 8
  // searches of a particle independent of each other (own cell: its
  // position); then the ranks, and each particle's number of candidates (ids
  // above its own in its partner cells)
  {
    int maxcnt = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) maxcnt = max(maxcnt, cb[d + 1] - cb[d]);
    int steps = 0;
    while ((1 << steps) <= maxcnt) ++steps;
    for (int k = t; k < nb; k += kEnumThreads) {
      const int32_t myid = sm.id[k];
      int pos[8], len[8];
#pragma unroll
      for (int d = 0; d < 8; ++d) { pos[d] = cb[d]; len[d] = cb[d + 1] - cb[d]; }
      for (int it = 0; it < steps; ++it) {
#pragma unroll
        for (int d = 0; d < 8; ++d) {
          const int half = len[d] >> 1;
          const bool below = len[d] > 0 && sm.id[pos[d] + half] < myid;
          pos[d] = below ? pos[d] + half + 1 : pos[d];
          len[d] = below ? len[d] - half - 1 : half;
        }
      }
#pragma unroll
      for (int d = 0; d < 8; ++d) sm.lb[k][d] = (uint8_t)(pos[d] - cb[d]);
    }
  }
  for (int q = t; q <= kMaxBlock; q += kEnumThreads) sm.hist[q] = 0;
  for (int d = 1 + t; d < nb; d += kEnumThreads)  // row d of the bitmap starts at F(nb - 1) - F(nb - d)
    sm.rowbase[d] = (uint16_t)(tri_f(nb - 1) - tri_f(nb - d));
  __syncthreads();
  for (int k = t; k < nb; k += kEnumThreads) {
    int r = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) r += sm.lb[k][d];
    sm.rank[k] = (uint8_t)r;
    sm.perm[r] = (uint8_t)k;
    const int dA = sm.code[k];
    const int free = 7 & ~(dA ^ (int)owner_bits(sm.id[k]));
    const int fixed = 7 & ~dA & ~free;
    int cand = 0, sub = free;
    for (;;) {
      const int dB = fixed | sub;
      cand += (sm.cbase[dB + 1] - sm.cbase[dB]) - (dB == dA ? sm.lb[k][dA] + 1 : sm.lb[k][dB]);
      if (sub == 0) break;
      sub = (sub - 1) & free;
    }
    sm.ncand[k] = (uint8_t)min(cand, 255);
    atomicAdd(&sm.hist[min(cand, 255)], 1);
  }
  __syncthreads();
  if (t < 32) {  // positions by candidate count, most first
    int run = 0;
    for (int l0 = 255; l0 >= 0; l0 -= 32) {
      const int l = l0 - lane;
      const int v = l >= 0 ? sm.hist[l] : 0;
      int incl = v;
#pragma unroll
      for (int sh = 1; sh < 32; sh <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, sh);
        if (lane >= sh) incl += u;
      }
      if (l >= 0) sm.hist[l] = run + incl - v;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  __syncthreads();
  for (int k = t; k < nb; k += kEnumThreads) sm.order[atomicAdd(&sm.hist[sm.ncand[k]], 1)] = (uint8_t)k;
  __syncthreads();
  // candidates: one thread per particle A (as the lower id), the particles
  // with the most candidates first, so that a warp's lanes have similar work
  const R h2 = (R)c.h2;
  for (int q = t; q < nb; q += kEnumThreads) {
    const int A = sm.order[q];
    const int dA = sm.code[A];
    const int hb = (int)owner_bits(sm.id[A]);
    const int free = 7 & ~(dA ^ hb);  // axes where the partner may share the cell
    const int fixed = 7 & ~dA & ~free;
    const int rA = sm.rank[A];
    const auto xa = sm.x[A];
    float4 fa = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (!P::mixed) fa = sm.f[A];
    const int wA = rA >> 5;
    const uint32_t bit = 1u << (rA & 31);
    int sub = free;
    for (;;) {
      const int dB = fixed | sub;
      const int b0 = dB == dA ? A + 1 : sm.cbase[dB] + sm.lb[A][dB], b1 = sm.cbase[dB + 1];
      for (int B = b0; B < b1; ++B) {
        if constexpr (!P::mixed) {  // float32 pre-test: skips only pairs with r >= h
          const float4 fb = sm.f[B];
          float ex = fa.x - fb.x, ey = fa.y - fb.y, ez = fa.z - fb.z;
          ex = ex > c.halfLf[0] ? ex - c.Lf[0] : (ex < -c.halfLf[0] ? ex + c.Lf[0] : ex);
          ey = ey > c.halfLf[1] ? ey - c.Lf[1] : (ey < -c.halfLf[1] ? ey + c.Lf[1] : ey);
          ez = ez > c.halfLf[2] ? ez - c.Lf[2] : (ez < -c.halfLf[2] ? ez + c.Lf[2] : ez);
          if (ex * ex + ey * ey + ez * ez >= c.h2_filter) continue;
        }
        const auto xb = sm.x[B];
        R dx, dy, dz;
        geo.disp((R)xa.x, (R)xa.y, (R)xa.z, (R)xb.x, (R)xb.y, (R)xb.z, dx, dy, dz);
        if (r2_of(dx, dy, dz) < h2) atomicOr(&sm.bits[sm.rowbase[sm.rank[B] - rA] + wA], bit);
      }
      if (sub == 0) break;
      sub = (sub - 1) & free;
    }
  }
  __syncthreads();
  // exclusive scan of the row populations (rows 1 .. nb - 1): each warp
  // scans 32 rows at a time, then the chunk totals are added in
  const int wid = t >> 5;
  for (int r0 = 1 + 32 * wid; r0 < nb; r0 += kEnumThreads) {
    const int rr = r0 + lane;
    int n = 0;
    if (rr < nb) {
      const int w0 = sm.rowbase[rr], nwr = (nb - rr + 31) >> 5;
      for (int w = 0; w < nwr; ++w) n += __popc(sm.bits[w0 + w]);
    }
    int incl = n;
#pragma unroll
    for (int sh = 1; sh < 32; sh <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, sh);
      if (lane >= sh) incl += v;
    }
    if (rr < nb) sm.rowoff[rr] = (uint16_t)(incl - n);  // within the chunk
    if (lane == 31) sm.hist[(r0 - 1) >> 5] = incl;        // chunk total
  }
  __syncthreads();
  if (t == 0) {  // chunk totals to chunk offsets (at most 8 chunks)
    int run = 0;
    for (int ch = 0; ch * 32 + 1 < nb; ++ch) {
      const int v = sm.hist[ch];
      sm.hist[ch] = run;
      run += v;
    }
    sm.npairs = run;
  }
  __syncthreads();
  for (int rr = 1 + t; rr < nb; rr += kEnumThreads) sm.rowoff[rr] = (uint16_t)(sm.rowoff[rr] + sm.hist[(rr - 1) >> 5]);
  __syncthreads();
  const int npairs = sm.npairs;
  if (npairs > kMaxPairs) {
    if (t == 0) hdr[o] = kHdrBig;
    return;
  }
  // write the pairs row by row (difference ascending), lower rank ascending
  uint16_t* out = canon + (int64_t)o * kMaxPairs;
  for (int rr = 1 + t; rr < nb; rr += kEnumThreads) {
    int pos = sm.rowoff[rr];
    const int w0 = sm.rowbase[rr], nwr = (nb - rr + 31) >> 5;
    for (int w = 0; w < nwr; ++w) {
      uint32_t bits = sm.bits[w0 + w];
      while (bits) {
        const int bit = __ffs(bits) - 1;
        bits &= bits - 1;
        const int lo = w * 32 + bit;
        out[pos++] = (uint16_t)(sm.perm[lo] | (sm.perm[lo + rr] << 8));
      }
    }
  }
  if (t == 0) hdr[o] = (uint32_t)npairs;
}

// Levels, step 1: one thread per block walks that block's canonical list and
// records the level of every pair (the longest chain of earlier pairs sharing
// a particle).  A warp handles 32 consecutive blocks and moves their lists
// and levels through shared memory 32 entries at a time, so every global
// access is coalesced.
constexpr int kLevelThreads = 32;
constexpr int kTile = 32;

__global__ void __launch_bounds__(kLevelThreads) k_sched_walk(int64_t ncell, int nc0, int nc1, int nc2,
                                                            uint32_t* __restrict__ hdr,
                                                            const uint16_t* __restrict__ canon,
                                                            uint8_t* __restrict__ level_of,
                                                            uint32_t* __restrict__ blk_hist,
                                                            const int32_t* __restrict__ cell_start,
                                                            const int32_t* __restrict__ mrank,
                                                            uint32_t* __restrict__ big_count,
                                                            int2* __restrict__ big_list) {
  __shared__ uint8_t last_s[kMaxBlock][kLevelThreads];  // level after which a particle is free
  __shared__ uint16_t tile[kLevelThreads][kTile + 1];
  __shared__ uint8_t ltile[kLevelThreads][kTile + 4];
  const int t = threadIdx.x;
  const int64_t o0 = (int64_t)blockIdx.x * kLevelThreads;
  const int64_t o = o0 + t;
  const bool live = o < ncell;
  const bool big = live && hdr[o] == kHdrBig;
  const int np = live && !big ? (int)(hdr[o] & 0xffffu) : 0;
  int npmax = np;
  for (int s = 16; s > 0; s >>= 1) npmax = max(npmax, __shfl_xor_sync(0xffffffffu, npmax, s));
  for (int k = 0; k < kMaxBlock; ++k) last_s[k][t] = 0;
  int nlev = 0;
  bool overflow = false;
  for (int k0 = 0; k0 < npmax; k0 += kTile) {
    // the next 32 entries of the 32 blocks' lists: all loads issued before
    // the first is used
    uint16_t v[kLevelThreads];
#pragma unroll
    for (int j = 0; j < kLevelThreads; ++j) {
      const int64_t oj = o0 + j;
      v[j] = oj < ncell ? canon[oj * kMaxPairs + k0 + t] : (uint16_t)0;
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < kLevelThreads; ++j) tile[j][t] = v[j];
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
#pragma unroll
    for (int j = 0; j < kLevelThreads; ++j) {
      const int64_t oj = o0 + j;
      if (oj < ncell) level_of[oj * kMaxPairs + k0 + t] = ltile[j][t];
    }
  }
  if (live) {
    // the block's colour is the parity pattern of its owner cell
    const int ox = (int)(o % nc0), oy = (int)((o / nc0) % nc1), oz = (int)(o / ((int64_t)nc0 * nc1));
    const int colour = (ox & 1) | ((oy & 1) << 1) | ((oz & 1) << 2);
    if (overflow || big) {
      // swept pair by pair after the colour's other blocks: listed with the
      // place of its particles in big_perm (blocks of a colour are disjoint)
      hdr[o] = kHdrBig;
      nlev = kMaxLevels;
      int nb = 0;
      for (int d = 0; d < 8; ++d) {
        int cx = ox + (d & 1), cy = oy + ((d >> 1) & 1), cz = oz + ((d >> 2) & 1);
        if (cx >= nc0) cx -= nc0;
        if (cy >= nc1) cy -= nc1;
        if (cz >= nc2) cz -= nc2;
        const int r = mrank[cx + nc0 * (cy + nc1 * cz)];
        nb += cell_start[r + 1] - cell_start[r];
      }
      const uint32_t off = atomicAdd(&big_count[8 + colour], (uint32_t)nb);
      const uint32_t slot = atomicAdd(&big_count[colour], 1u);
      big_list[colour * (ncell >> 3) + slot] = make_int2((int)o, (int)off);
    } else {
      hdr[o] = (uint32_t)np | ((uint32_t)nlev << 16);
    }
    atomicAdd(&blk_hist[colour * 256 + nlev], 1u);
  }
}

// ---------------------------------------------------------------------------
// The order in which a colour launch hands out its blocks: deepest first.
// Each warp of a colour launch runs its blocks in lockstep and pays for the
// deepest, so neighbours in this order have similar depth, and the deep
// blocks start first, which keeps the launch's tail short.  Blocks of a colour
// are independent, so the order changes no result.
// Step 1 (8 thread blocks of 256, one per colour): the depth histogram turned
// into each depth's first position, deepest first.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sched_order_scan(uint32_t* __restrict__ blk_hist) {
  __shared__ uint32_t warp_sum[8];
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  uint32_t* h = blk_hist + blockIdx.x * 256;
  const uint32_t v = h[255 - t];  // thread t takes depth 255 - t
  uint32_t incl = v;
#pragma unroll
  for (int sh = 1; sh < 32; sh <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, sh);
    if (lane >= sh) incl += x;
  }
  if (lane == 31) warp_sum[wp] = incl;
  __syncthreads();
  uint32_t before = 0;
  for (int k = 0; k < wp; ++k) before += warp_sum[k];
  __syncthreads();
  h[255 - t] = before + incl - v;
}

// Step 2 (one thread per owner cell): each block's place in its colour's
// order, by depth; the order among blocks of equal depth is free.
__global__ void k_sched_order_scatter(int64_t ncell, int nc0, int nc1, const uint32_t* __restrict__ hdr,
                                      uint32_t* __restrict__ blk_hist, int32_t* __restrict__ blk_order) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= ncell) return;
  const int ox = (int)(o % nc0), oy = (int)((o / nc0) % nc1), oz = (int)(o / ((int64_t)nc0 * nc1));
  const int colour = (ox & 1) | ((oy & 1) << 1) | ((oz & 1) << 2);
  const int hx = nc0 >> 1, hy = nc1 >> 1;
  const int32_t w = (ox >> 1) + hx * ((oy >> 1) + hy * (oz >> 1));  // index among the colour's blocks
  const uint32_t hd = hdr[o];
  const int nlev = hd == kHdrBig ? kMaxLevels : (int)(hd >> 16);
  const uint32_t pos = atomicAdd(&blk_hist[colour * 256 + nlev], 1u);
  blk_order[colour * (ncell >> 3) + pos] = w;
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
  if (hd == kHdrBig) return;
  const int np = (int)(hd & 0xffffu), nlev = (int)(hd >> 16);
  int32_t* cnt = cnt_s[warp];
  for (int L = lane; L <= kMaxLevels; L += 32) cnt[L] = 0;
  __syncwarp();
  const uint16_t* in = canon + o * kMaxPairs;
  const uint8_t* lv = level_of + o * kMaxPairs;
#pragma unroll 4
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
#pragma unroll 4
  for (int k = lane; k < np; k += 32) out[atomicAdd(&cnt[lv[k]], 1)] = in[k];
}


template <class P>
void launch_fd_schedule(const Consts& c, const Workspace& w, int cur, cudaStream_t s) {
  if (c.N == 0) return;
  Arrays<P> a = view<P>(w, cur);
  uint16_t* canon = w.sched_pair + (size_t)c.ncell * kMaxPairs;
  k_sched_enum<P><<<(unsigned)c.ncell, kEnumThreads, 0, s>>>(c, a, w.cell_start, w.mrank, w.xmin[0], w.xmin[1],
                                                               w.xmin[2], w.qf4, w.sched_hdr, canon, w.blk_hist,
                                                               w.big_count);
  k_sched_walk<<<(unsigned)((c.ncell + kLevelThreads - 1) / kLevelThreads), kLevelThreads, 0, s>>>(
      c.ncell, c.nc[0], c.nc[1], c.nc[2], w.sched_hdr, canon, w.level_of, w.blk_hist, w.cell_start, w.mrank,
      w.big_count, w.big_list);
  k_sched_bucket<<<(unsigned)((c.ncell + kBucketWarps - 1) / kBucketWarps), kBucketWarps * 32, 0, s>>>(
      c.ncell, w.sched_hdr, canon, w.level_of, w.sched_lvl, w.sched_pair);
  k_sched_order_scan<<<8, 256, 0, s>>>(w.blk_hist);
  k_sched_order_scatter<<<(unsigned)((c.ncell + 255) / 256), 256, 0, s>>>(c.ncell, c.nc[0], c.nc[1], w.sched_hdr,
                                                                         w.blk_hist, w.blk_order);
}

__global__ void k_sweep_set(unsigned long long* sweep, unsigned long long v) { *sweep = v; }
__global__ void k_sweep_advance(unsigned long long* sweep) { *sweep += 1ull; }

void launch_set_sweep(const Workspace& w, unsigned long long value, cudaStream_t s) {
  k_sweep_set<<<1, 1, 0, s>>>(w.sweep, value);
}
void launch_advance_sweep(const Workspace& w, cudaStream_t s) { k_sweep_advance<<<1, 1, 0, s>>>(w.sweep); }

template void launch_fd_schedule<Fp64>(const Consts&, const Workspace&, int, cudaStream_t);
template void launch_fd_schedule<Mixed>(const Consts&, const Workspace&, int, cudaStream_t);

}  // namespace sdpd
