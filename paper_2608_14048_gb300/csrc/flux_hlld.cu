// Flux pass instantiations: adiabatic HLLD (Miyoshi & Kusano 2005).
#include "flux3.cuh"

namespace aeth {

template <typename R, bool P64, bool MHD, int SOLVER, bool DUAL>
void flux_pass_solver(aeth_ctx* c, int recon, int src, int block) {
  flux_pass_solver_impl<R, P64, MHD, SOLVER, DUAL>(c, recon, src, block);
}

#define AETH_FLUX_INST(R, P64)                                               \
  template void flux_pass_solver<R, P64, true, 0>(aeth_ctx*, int, int, int); \
  template void flux_pass_solver<R, P64, false, 0>(aeth_ctx*, int, int, int);
AETH_FLUX_INST(float, false)
AETH_FLUX_INST(float, true)
AETH_FLUX_INST(double, false)
#undef AETH_FLUX_INST

}  // namespace aeth
