// render_shaded.cu -- the shaded ray marchers: gradient shading (R13) and
// opacity correction (R14), the second render workload.  Same traversals and
// sample lattice as render.cu; only the per-sample colour and opacity differ.
#include "render_kernels.h"

namespace ess {

template void launch_render_kernels<1>(Ctx &, const RArgs &, int, ess_dtype, int);
template void launch_batch_kernels<1>(Ctx &, int, ess_dtype, bool, bool, const RArgs *, const int *,
                                      BatchHeader *);

}  // namespace ess
