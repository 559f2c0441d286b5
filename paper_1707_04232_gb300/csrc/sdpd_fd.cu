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
// positions only, which are fixed during the sweep): k_sched_enum (one
// thread block per block: owned pairs in canonical order, from the
// neighbour lists of the density pass), k_sched_walk (one thread per
// block: the dependency level of every pair) and k_sched_bucket (one warp per
// block: pairs bucketed by level); two more order each colour's blocks by
// depth (k_sched_order_scan, k_sched_order_scatter); then k_fd_colour (sdpd_fd_colour.cuh)
// runs once per colour: the pair updates level by level in shared memory,
// one or two blocks per warp as the launch's block schedule says.
#include "sdpd_fd_common.cuh"

namespace sdpd {


// ---------------------------------------------------------------------------
// Schedule, step 1: owned pairs of every block in canonical order, read from
// the neighbour lists of the density pass.  One thread block of
// kEnumThreads threads per owner cell.
// Owned pairs.  The pairs of this block whose lower id is particle A (block
// cell dA) are A's neighbours in the cells that this block holds and that
// the owner rule gives to this block when A is the lower id: per axis k the
// offset +1 (A's cell is the block's lower one: dA_k = 0) or -1 (its upper
// one), and the offset 0 where bit k of A's owner bits equals dA_k.  These
// cells are 1, 2 or 4 rows of A's 27-cell walk, each a run of consecutive
// cells, so their entries are at most four slot ranges of A's list (the
// density pass records where each row's cells start and end).  Of these
// entries, those whose partner ranks above A are A's owned pairs; the others
// are found from the partner's side.  The predicate is the density pass's
// r^2 < h^2, so the sweep's pair set is the one of the density sum.  A block
// with a member whose list overflowed its row is swept pair by pair
// (kHdrBig).
// Ranks.  Every cell holds its particles by ascending id; the 8 sorted cells
// are merged in three rounds of pairwise merges (the place of an id in the
// merged run = its place in its own run + the ids below it in the sibling
// run, by binary search), which gives each particle's rank among the block's
// ids and the particle of each rank.
// Entries.  The members' entry counts are scanned into offsets of one flat
// range, and the threads take its entries in turn, so that the global loads
// are spread evenly and issued together (in chunks of kFlatEntries, the
// size of the table of each entry's member).
// Found pairs set bit rank(i) of row d = rank(j) - rank(i) of a triangular
// bitmap (row d holds nb - d bits in whole words: it starts at word
// F(nb - 1) - F(nb - d) with F(n) = sum_{k <= n} ceil(k / 32)), which is then
// read out row by row.
// ---------------------------------------------------------------------------
constexpr int kEnumThreads = 160;
constexpr int kEnumWarps = kEnumThreads / 32;
constexpr int kTriWords = 1152;   // >= F(255) = 1144: a triangle of 256 rows
constexpr int kFlatEntries = 2048;  // group entries of one block per chunk

// words of the first rows of the triangular bitmap: F(n) = sum_{k=1..n} ceil(k/32)
__device__ __forceinline__ int tri_f(int n) {
  const int q = n >> 5, s = n & 31;
  return 16 * q * (q + 1) + s * (q + 1);
}

struct EnumSmem {
  uint32_t bits[kTriWords];
  int32_t ids[2][kMaxBlock];  // merge rounds: the ids in run order
  uint8_t ks[2][kMaxBlock];   // and the block-local index of each
  uint8_t rank[kMaxBlock];    // rank of each block-local index
  uint8_t perm[kMaxBlock];    // block-local index of each rank
  uint8_t who[kFlatEntries];  // member of each flat entry
  uint32_t rng[kMaxBlock];    // up to four slot ranges (first slot, length) of each member's group, packed
  uint32_t rcum[kMaxBlock];   // cumulative lengths after ranges 0, 1, 2 (bytes)
  uint8_t ncnt[kMaxBlock];    // entries of each member's group
  uint8_t dk[kMaxBlock];      // block cell of each member
  int64_t lbase[kMaxBlock];   // nbr_slot(member, 0) with the slot's in-row part removed
  uint8_t dtab[8][64];        // partner cell of (member cell, stencil code); 8: not in the block
  int32_t off[kMaxBlock + 1];  // first flat entry of each member
  uint16_t rowbase[kMaxBlock];  // first word of each row of the bitmap
  int32_t wtot[kEnumWarps];     // per-warp totals of the offset scan
  int32_t ctot[8];              // row-scan chunk totals
  int32_t cstart[8], cbase[9], koff[9];
  int32_t nb, big;
};

__global__ void __launch_bounds__(kEnumThreads)
    k_sched_enum(Consts c, const int32_t* __restrict__ pid, const int32_t* __restrict__ cell_start,
                 const int32_t* __restrict__ mrank, const uint32_t* __restrict__ nlist,
                 const int32_t* __restrict__ nn, const uint32_t* __restrict__ cend, uint32_t* __restrict__ hdr,
                 uint16_t* __restrict__ canon, uint32_t* __restrict__ blk_hist, uint32_t* __restrict__ big_count) {
  __shared__ EnumSmem sm;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
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
      sm.koff[lane] = cinc - ccnt - cst;  // block-local index = storage index + koff
    }
    if (lane == 7) {
      sm.cbase[8] = cinc;
      sm.nb = cinc;
    }
    if (lane == 0) {
      sm.big = 0;
      sm.koff[8] = -(1 << 30);  // a partner outside the block: out of range
    }
  }
  for (int q = t; q < 8 * 64; q += kEnumThreads) {  // partner cell: member cell + (code - 1) per axis
    const int dA = q >> 6, code = q & 63;
    int dB = 0;
    bool in = true;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int f = (code >> (2 * ax)) & 3, b = ((dA >> ax) & 1) + f - 1;
      in = in && f < 3 && b >= 0 && b <= 1;
      dB |= (b & 1) << ax;
    }
    sm.dtab[dA][code] = (uint8_t)(in ? dB : 8);
  }
  __syncthreads();
  const int nb = sm.nb;
  if (nb > kMaxBlock) {  // beyond capacity: swept pair by pair (see kHdrBig)
    if (t == 0) hdr[o] = kHdrBig;
    return;
  }
  const int ntri = nb > 1 ? tri_f(nb - 1) : 0;  // words of the bitmap in use
  for (int q = t; q < ntri; q += kEnumThreads) sm.bits[q] = 0u;
  int cb[9];
#pragma unroll
  for (int u = 0; u < 9; ++u) cb[u] = sm.cbase[u];
  const int64_t N = c.N;
  // the members: id, and the slot ranges of the owner group in the list
  for (int k = t; k < nb; k += kEnumThreads) {
    int d = 0;
#pragma unroll
    for (int u = 1; u < 8; ++u) d += (k >= cb[u]);
    const int g = sm.cstart[d] + (k - sm.cbase[d]);
    const int32_t id = __ldg(&pid[g]);
    sm.ids[0][k] = id;
    sm.ks[0][k] = (uint8_t)k;
    if (__ldg(&nn[g]) > c.nbr_cap) sm.big = 1;  // the list lost entries
    const unsigned ob = owner_bits(id);
    // per axis the cells of the group as indices [lo, hi) of the offsets
    // (-1, 0, +1): dA_k = 0: {0 if ob_k = 0, +1}; dA_k = 1: {-1, 0 if ob_k = 1}
    int lo[3], hi[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int dk = (d >> ax) & 1, bk = (int)(ob >> ax) & 1;
      lo[ax] = dk ? 0 : 2 - (bk ^ 1);
      hi[ax] = dk ? 1 + bk : 3;
    }
    // rows (iz, iy) of the group: at most 2 x 2; x range [lo[0], hi[0]) of bytes
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int iz = lo[2] + (q >> 1), iy = lo[1] + (q & 1);
      w[q] = (iz < hi[2] && iy < hi[1]) ? __ldg(&cend[(int64_t)(iz * 3 + iy) * N + g]) : 0u;
    }
    uint32_t rng = 0u, cum = 0u;
    int tot = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s0 = (int)((w[q] >> (8 * lo[0])) & 255u), s1 = (int)((w[q] >> (8 * hi[0])) & 255u);
      const int len = s1 > s0 ? s1 - s0 : 0;  // empty for rows outside the group (w = 0)
      rng |= (uint32_t)s0 << (8 * q);
      tot += len;
      if (q < 3) cum |= (uint32_t)min(tot, 255) << (8 * q);
    }
    sm.rng[k] = rng;
    sm.rcum[k] = cum;
    sm.off[k] = tot;  // the count; turned into an offset below
    sm.ncnt[k] = (uint8_t)tot;  // at most the row capacity
    sm.dk[k] = (uint8_t)d;
    sm.lbase[k] = ((int64_t)(g >> 5) * (c.nbr_cap >> 2) << 7) + ((g & 31) << 2);
  }
  __syncthreads();
  if (sm.big) {
    if (t == 0) hdr[o] = kHdrBig;
    return;
  }
  // the member of each flat entry of the chunk [E0, E0 + kFlatEntries), in
  // equal stretches per thread: one binary search for the stretch's first
  // entry, then a walk (members without entries are skipped)
  auto fill_who = [&](int E0) {
    const int E = sm.off[nb], Ec = min(E - E0, kFlatEntries), per = (Ec + kEnumThreads - 1) / kEnumThreads;
    const int e0 = E0 + t * per, e1 = min(E0 + Ec, e0 + per);
    if (e0 < e1) {
      int pos = 1, len = nb - 1;  // members 1 .. nb - 1 starting at or before e0
      while (len > 0) {
        const int half = len >> 1;
        const bool le = sm.off[pos + half] <= e0;
        pos = le ? pos + half + 1 : pos;
        len = le ? len - half - 1 : half;
      }
      int k = pos - 1, kend = sm.off[k] + sm.ncnt[k];
      for (int e = e0; e < e1; ++e) {
        while (e >= kend) {
          ++k;
          kend = sm.off[k] + sm.ncnt[k];
        }
        sm.who[e - E0] = (uint8_t)k;
      }
    }
  };
  // ranks: three rounds of pairwise merges of the sorted cells, interleaved
  // with the exclusive scan of the members' entry counts
  int cnt0 = 0, incl = 0;
#pragma unroll 1
  for (int L = 0; L < 3; ++L) {
    const int src = L & 1, dst = src ^ 1;
    for (int k = t; k < nb; k += kEnumThreads) {
      const int d = sm.dk[k];
      const int run = d >> L, sib = run ^ 1;
      const int own0 = sm.cbase[run << L], m0 = sm.cbase[(run & ~1) << L];
      int pos = sm.cbase[sib << L], len = sm.cbase[(sib + 1) << L] - pos;
      const int sib0 = pos;
      const int32_t myid = sm.ids[src][k];
      while (len > 0) {
        const int half = len >> 1;
        const bool below = sm.ids[src][pos + half] < myid;
        pos = below ? pos + half + 1 : pos;
        len = below ? len - half - 1 : half;
      }
      const int np = m0 + (k - own0) + (pos - sib0);
      sm.ids[dst][np] = myid;
      sm.ks[dst][np] = sm.ks[src][k];
    }
    if (L == 0) {  // counts of members 2t and 2t + 1: per-warp inclusive scan
      cnt0 = 2 * t < nb ? sm.ncnt[2 * t] : 0;
      const int cnt1 = 2 * t + 1 < nb ? sm.ncnt[2 * t + 1] : 0;
      incl = cnt0 + cnt1;
#pragma unroll
      for (int sh = 1; sh < 32; sh <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, sh);
        if (lane >= sh) incl += v;
      }
      if (lane == 31) sm.wtot[wid] = incl;
    } else if (L == 1) {  // offsets in member order
      int before = 0, total = 0;
#pragma unroll
      for (int q = 0; q < kEnumWarps; ++q) {
        before += q < wid ? sm.wtot[q] : 0;
        total += sm.wtot[q];
      }
      const int ex = before + incl - cnt0 - (2 * t + 1 < nb ? sm.ncnt[2 * t + 1] : 0);
      if (2 * t < nb) sm.off[2 * t] = ex;
      if (2 * t + 1 < nb) sm.off[2 * t + 1] = ex + cnt0;
      if (t == 0) sm.off[nb] = total;
    } else {  // the member of each entry of the first chunk
      fill_who(0);
    }
    __syncthreads();
  }
  for (int r = t; r < nb; r += kEnumThreads) {  // the merged run is ids[1]
    const int k = sm.ks[1][r];
    sm.perm[r] = (uint8_t)k;
    sm.rank[k] = (uint8_t)r;
  }
  for (int d = 1 + t; d < nb; d += kEnumThreads)  // row d of the bitmap starts at F(nb - 1) - F(nb - d)
    sm.rowbase[d] = (uint16_t)(tri_f(nb - 1) - tri_f(nb - d));
  __syncthreads();
  // the flat entries: partner, rank test, bit; chunk by chunk (a block with
  // more entries than the table holds takes several)
  const int E = sm.off[nb];
  for (int E0 = 0; E0 < E; E0 += kFlatEntries) {
    if (E0 > 0) {
      fill_who(E0);
      __syncthreads();
    }
    const int E1 = min(E, E0 + kFlatEntries);
#pragma unroll 4
    for (int e = E0 + t; e < E1; e += kEnumThreads) {
      const int A = sm.who[e - E0];
      const int m = e - sm.off[A];
      const uint32_t rng = sm.rng[A], cum = sm.rcum[A];
      const int c0 = cum & 255u, c1 = (cum >> 8) & 255u, c2 = (cum >> 16) & 255u;
      const int q = (m >= c0) + (m >= c1) + (m >= c2);
      const int before = q == 0 ? 0 : (q == 1 ? c0 : (q == 2 ? c1 : c2));
      const int slot = (int)((rng >> (8 * q)) & 255u) + (m - before);
      const int dA = sm.dk[A];
      const uint32_t en = __ldg(&nlist[sm.lbase[A] + ((slot >> 2) << 7) + (slot & 3)]);  // nbr_slot(g, slot)
      const int kB = (int)(en >> 6) + sm.koff[sm.dtab[dA][en & 63u]];
      if ((unsigned)kB < (unsigned)nb) {
        const int rA = sm.rank[A], rB = sm.rank[kB];
        if (rB > rA) atomicOr(&sm.bits[sm.rowbase[rB - rA] + (rA >> 5)], 1u << (rA & 31));
      }
    }
    __syncthreads();
  }
  // row populations (rows 1 .. nb - 1): each warp scans 32 rows at a time
  // (row 1 + t is thread t's in every phase below), then the chunk totals
  // are added in
  int rowex[2] = {0, 0};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int r0 = 1 + 32 * wid + it * kEnumThreads;
    if (r0 >= nb) break;
    const int rr = r0 + lane;
    int n = 0;
    if (rr < nb) {
      const int w0 = sm.rowbase[rr], nwr = (nb - rr + 31) >> 5;
      for (int w = 0; w < nwr; ++w) n += __popc(sm.bits[w0 + w]);
    }
    int inc = n;
#pragma unroll
    for (int sh = 1; sh < 32; sh <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, sh);
      if (lane >= sh) inc += v;
    }
    rowex[it] = inc - n;
    if (lane == 31) sm.ctot[(r0 - 1) >> 5] = inc;
  }
  __syncthreads();
  const int nchunk = (nb - 1 + 31) >> 5;
  int npairs = 0;
  for (int ch = 0; ch < nchunk; ++ch) npairs += sm.ctot[ch];
  if (npairs > kMaxPairs) {
    if (t == 0) hdr[o] = kHdrBig;
    return;
  }
  // write the pairs row by row (difference ascending), lower rank ascending
  uint16_t* out = canon + (int64_t)o * kMaxPairs;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int rr = 1 + t + it * kEnumThreads;
    if (rr >= nb) break;
    const int chunk = (rr - 1) >> 5;
    int pos = rowex[it];
    for (int ch = 0; ch < chunk; ++ch) pos += sm.ctot[ch];
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
  k_sched_enum<<<(unsigned)c.ncell, kEnumThreads, 0, s>>>(c, a.id, w.cell_start, w.mrank, w.nlist, w.nn, w.cend,
                                                          w.sched_hdr, canon, w.blk_hist, w.big_count);
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
