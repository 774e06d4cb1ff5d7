// Flux pass instantiations: the face-state dump of the learned flux (the
// reconstructed states are written out for the network instead of solved).
#include "flux3.cuh"

namespace aeth {

template <typename R, bool P64, bool MHD, int SOLVER, bool DUAL>
void flux_pass_solver(aeth_ctx* c, int recon, int src, int block) {
  flux_pass_solver_impl<R, P64, MHD, SOLVER, DUAL>(c, recon, src, block);
}

#define AETH_FLUX_INST(R, P64, S)                                            \
  template void flux_pass_solver<R, P64, true, S>(aeth_ctx*, int, int, int); \
  template void flux_pass_solver<R, P64, false, S>(aeth_ctx*, int, int, int);
AETH_FLUX_INST(float, false, 1)
AETH_FLUX_INST(float, true, 1)
AETH_FLUX_INST(double, false, 1)
#undef AETH_FLUX_INST

}  // namespace aeth
