// sdpd_stats.cu -- statistics of the internal energies on the device: the
// histogram from which the distribution of eps is compared with the Gamma
// marginal of the ideal gas, Eq. (dist-analytic), and its error, Eq.
// (error-dist), in FD-only runs.
#include "sdpd_internal.cuh"

namespace sdpd {

namespace {

// Per-block histogram in shared memory, then one atomic add per bin.
// Bin b of nbins holds lo + b w <= x < lo + (b + 1) w with x = eps * scale
// and b = floor((x - lo) / w) capped at nbins - 1; slot nbins counts x < lo,
// slot nbins + 1 counts x >= hi and non-finite x.
__global__ void __launch_bounds__(256) k_energy_hist(int64_t N, const double* __restrict__ eps, double scale,
                                                     double lo, double hi, double w, int nbins,
                                                     unsigned long long* __restrict__ counts) {
  extern __shared__ unsigned int bins[];
  for (int b = threadIdx.x; b < nbins + 2; b += blockDim.x) bins[b] = 0u;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = __dmul_rn(eps[i], scale);
    int b;
    if (x < lo) {
      b = nbins;
    } else if (!(x < hi)) {
      b = nbins + 1;
    } else {
      const double t = __ddiv_rn(__dsub_rn(x, lo), w);
      b = min((int)floor(t), nbins - 1);
    }
    atomicAdd(&bins[b], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins + 2; b += blockDim.x)
    if (bins[b]) atomicAdd(&counts[b], (unsigned long long)bins[b]);
}

}  // namespace

void launch_energy_hist(const Consts& c, const Workspace& w, int cur, double lo, double hi, int nbins,
                        double scale, unsigned long long* counts, cudaStream_t s) {
  if (c.N == 0) return;
  const double wbin = (hi - lo) / (double)nbins;
  const unsigned blocks = (unsigned)std::min<int64_t>((c.N + 255) / 256, 4 * 152);
  k_energy_hist<<<blocks, 256, (size_t)(nbins + 2) * sizeof(unsigned int), s>>>(c.N, w.eps[cur], scale, lo, hi,
                                                                                  wbin, nbins, counts);
}

}  // namespace sdpd
