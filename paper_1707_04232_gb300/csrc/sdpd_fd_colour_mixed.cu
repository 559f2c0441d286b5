// sdpd_fd_colour_mixed.cu -- the colour kernels of the mixed-precision path, every
// block-schedule variant (kept apart from the other precision so that the
// variants compile in parallel).
#include "sdpd_fd_colour.cuh"

namespace sdpd {

template void fd_prepare<Mixed, Mixed>();
template void launch_fd_colours<Mixed, Mixed>(const Consts&, const Workspace&, int, double, uint64_t, int,
                                    cudaStream_t);

}  // namespace sdpd
