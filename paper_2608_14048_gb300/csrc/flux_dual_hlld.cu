// Flux pass instantiations with the dual-energy formalism (Sec. 2.8):
// HLLD plus the upwinded entropy flux, FP64 and FP32.
#include "flux3.cuh"

namespace aeth {

template <typename R, bool P64, bool MHD, int SOLVER, bool DUAL>
void flux_pass_solver(aeth_ctx* c, int recon, int src, int block) {
  flux_pass_solver_impl<R, P64, MHD, SOLVER, DUAL>(c, recon, src, block);
}

#define AETH_FLUX_INST(R)                                                          \
  template void flux_pass_solver<R, false, true, 0, true>(aeth_ctx*, int, int, int); \
  template void flux_pass_solver<R, false, false, 0, true>(aeth_ctx*, int, int, int);
AETH_FLUX_INST(float)
AETH_FLUX_INST(double)
#undef AETH_FLUX_INST

}  // namespace aeth
