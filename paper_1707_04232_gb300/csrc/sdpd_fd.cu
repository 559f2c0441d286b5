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
  // the partner segments of the 32 particles of the current chunk, one row
  // per lane: entries before segment s (cum, 0xff past the last), and the
  // segment's first entry and partner cell (first | cell << 8)
  uint8_t seg_cum[32][8];
  uint16_t seg_pk[32][8];
};

// The owned pairs are read from the neighbour lists of the density pass: as
// the lower id of a pair, a particle in block cell dA has owned partners only
// in the cells dB that agree with dA exactly where dA agrees with its owner
// bits (and differ from dA elsewhere), whose entries sit in known stencil
// groups of its list row; entries with a lower-ranked partner belong to the
// partner's side.  Over the 8 blocks holding a particle these groups cover
// its list once.
template <class P>
__global__ void __launch_bounds__(kSchedWarps * 32)
    k_sched_enum(Consts c, Arrays<P> a, const int32_t* __restrict__ cell_start, const int32_t* __restrict__ mrank,
                 const uint32_t* __restrict__ nlist, const uint8_t* __restrict__ nbr_off,
                 uint32_t* __restrict__ hdr, uint16_t* __restrict__ canon, int* status,
                 uint32_t* __restrict__ blk_hist) {
  __shared__ SchedSmem sm_all[kSchedWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (blockIdx.x == 0)  // the depth histogram that k_sched_walk fills
    for (int k = threadIdx.x; k < 8 * 256; k += blockDim.x) blk_hist[k] = 0u;
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
  // Owned entries, spread over the warp: each lane lists the partner
  // segments of one particle of a chunk of 32, a warp prefix sum over the
  // lanes' entry totals maps the chunk's entries to lanes, and each entry
  // finds its segment in the owner lane's row, so that the lanes load
  // consecutive entries of a row together and share the work evenly (a
  // particle has from one to eight partner segments, ~3 to ~80 entries).
  for (int k0 = 0; k0 < nb; k0 += 32) {
    const int k = k0 + lane;
    const bool live = k < nb;
    int dA = 0, g = 0, rk = 0;
    if (live) {
      dA = code_of(k);
      g = sm.cstart[dA] + (k - sm.cbase[dA]);
      rk = sm.rank[k];
    }
    // Partner cells of a pair this block owns with k as the lower id: along
    // an axis where k's block-cell bit equals k's owner bit the partner may
    // share the coordinate or sit across (free axes); elsewhere it must sit
    // across.
    const int hb = live ? (int)owner_bits(sm.id[k]) : 0;
    const int free = 7 & ~(dA ^ hb);
    const int fixed = 7 & ~dA & ~free;
    int tot = 0, ns = 0;
    if (live) {
      const uint8_t* off = nbr_off + (int64_t)g * 28;
      int sub = free;
      for (;;) {  // partner cells dB = fixed | (subsets of free)
        const int dB = fixed | sub;
        const int sx = ((dB & 1) - (dA & 1)) + 1, sy = (((dB >> 1) & 1) - ((dA >> 1) & 1)) + 1,
                  sz = (((dB >> 2) & 1) - ((dA >> 2) & 1)) + 1;
        const int st = sx + 3 * sy + 9 * sz;
        const int e0 = off[st], n = off[st + 1] - e0;
        if (n > 0) {
          sm.seg_cum[lane][ns] = (uint8_t)tot;
          sm.seg_pk[lane][ns] = (uint16_t)(e0 | (dB << 8));
          tot += n;
          ++ns;
        }
        if (sub == 0) break;
        sub = (sub - 1) & free;
      }
    }
    for (int t = ns; t < 8; ++t) sm.seg_cum[lane][t] = 0xff;
    __syncwarp();
    int incl = tot;
#pragma unroll
    for (int sh = 1; sh < 32; sh <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, sh);
      if (lane >= sh) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - tot;
    // kDeep rounds of 32 entries per iteration, all list loads issued before
    // any is used
    constexpr int kDeep = 4;
    for (int t0 = 0; t0 < total; t0 += 32 * kDeep) {
      int o_rk[kDeep], o_q[kDeep], o_b[kDeep];
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
        const int o_ex = __shfl_sync(0xffffffffu, excl, src);
        const int o_g = __shfl_sync(0xffffffffu, g, src);
        o_rk[h] = __shfl_sync(0xffffffffu, rk, src);
        o_q[h] = -1;
        o_b[h] = 0;
        if (t < total) {
          const int u = t - o_ex;  // entry of the owner lane's particle
          int sg = 0;
#pragma unroll
          for (int s2 = 1; s2 < 8; ++s2) sg += (int)sm.seg_cum[src][s2] <= u;
          const int pk = sm.seg_pk[src][sg];
          o_q[h] = (pk & 255) + (u - sm.seg_cum[src][sg]);
          o_b[h] = pk >> 8;
        }
        ent[h] = o_q[h] >= 0 ? __ldg(&nlist[(int64_t)o_g * c.nbr_cap + o_q[h]]) : 0u;
      }
#pragma unroll
      for (int h = 0; h < kDeep; ++h) {
        if (o_q[h] >= 0) {
          const int oB = o_b[h];
          const int j = (int)(ent[h] >> 6);
          const int rj = sm.rank[sm.cbase[oB] + (j - sm.cstart[oB])];
          if (o_rk[h] < rj) atomicOr(&sm.bits[o_rk[h] >> 5][rj - o_rk[h]], 1u << (o_rk[h] & 31));
        }
      }
    }
    __syncwarp();  // the segment rows are refilled by the next chunk
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

__global__ void __launch_bounds__(kLevelThreads) k_sched_walk(int64_t ncell, int nc0, int nc1,
                                                            uint32_t* __restrict__ hdr,
                                                            const uint16_t* __restrict__ canon,
                                                            uint8_t* __restrict__ level_of, int* status,
                                                            uint32_t* __restrict__ blk_hist) {
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
      nlev = 0;
    } else {
      hdr[o] = (uint32_t)np | ((uint32_t)nlev << 16);
    }
    // the block's colour is the parity pattern of its owner cell
    const int ox = (int)(o % nc0), oy = (int)((o / nc0) % nc1), oz = (int)(o / ((int64_t)nc0 * nc1));
    const int colour = (ox & 1) | ((oy & 1) << 1) | ((oz & 1) << 2);
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
  const int nlev = (int)(hdr[o] >> 16);
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


template <class P>
void launch_fd_schedule(const Consts& c, const Workspace& w, int cur, cudaStream_t s) {
  if (c.N == 0) return;
  Arrays<P> a = view<P>(w, cur);
  uint16_t* canon = w.sched_pair + (size_t)c.ncell * kMaxPairs;
  const unsigned gs = (unsigned)((c.ncell + kSchedWarps - 1) / kSchedWarps);
  k_sched_enum<P><<<gs, kSchedWarps * 32, 0, s>>>(c, a, w.cell_start, w.mrank, w.nlist, w.nbr_off,
                                                   w.sched_hdr, canon, w.status, w.blk_hist);
  k_sched_walk<<<(unsigned)((c.ncell + kLevelThreads - 1) / kLevelThreads), kLevelThreads, 0, s>>>(
      c.ncell, c.nc[0], c.nc[1], w.sched_hdr, canon, w.level_of, w.status, w.blk_hist);
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
