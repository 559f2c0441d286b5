// sdpd_fd_colour_fp64.cu -- the colour kernels of the float64 state, every
// block-schedule variant, with float64 or float32 pair arithmetic (kept apart
// from the mixed state so that the variants compile in parallel).
#include "sdpd_fd_colour.cuh"

namespace sdpd {

template void fd_prepare<Fp64, Fp64>();
template void fd_prepare<Fp64, Mixed>();
template void launch_fd_colours<Fp64, Fp64>(const Consts&, const Workspace&, int, double, uint64_t, int,
                                          cudaStream_t);
// float64 state, float32 pair arithmetic
template void launch_fd_colours<Fp64, Mixed>(const Consts&, const Workspace&, int, double, uint64_t, int,
                                           cudaStream_t);

template <class P, int V>
constexpr bool fits_v() { return fd_fits<P, kFdOpw[V], kFdWarps[V]>(); }

bool fd_variant_fits(bool mixed, int v) {
  switch (v) {
    case 0: return mixed ? fits_v<Mixed, 0>() : fits_v<Fp64, 0>();
    case 1: return mixed ? fits_v<Mixed, 1>() : fits_v<Fp64, 1>();
    case 2: return mixed ? fits_v<Mixed, 2>() : fits_v<Fp64, 2>();
    case 3: return mixed ? fits_v<Mixed, 3>() : fits_v<Fp64, 3>();
    case 4: return mixed ? fits_v<Mixed, 4>() : fits_v<Fp64, 4>();
    default: return false;
  }
}

}  // namespace sdpd
