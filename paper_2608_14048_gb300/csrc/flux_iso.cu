// Flux pass instantiations: isothermal closure p = cs^2 rho with the
// isothermal HLLD (Mignone 2007) and HLLE solvers.  The isothermal pressure
// needs no FP64 energy difference, so the FP32 path serves both FP32 modes.
#include "flux3.cuh"

namespace aeth {

template <typename R, bool P64, bool MHD, int SOLVER, bool DUAL>
void flux_pass_solver(aeth_ctx* c, int recon, int src, int block) {
  flux_pass_solver_impl<R, P64, MHD, SOLVER, DUAL>(c, recon, src, block);
}

#define AETH_FLUX_INST(R, S)                                                   \
  template void flux_pass_solver<R, false, true, S>(aeth_ctx*, int, int, int); \
  template void flux_pass_solver<R, false, false, S>(aeth_ctx*, int, int, int);
AETH_FLUX_INST(float, 3)
AETH_FLUX_INST(float, 4)
AETH_FLUX_INST(double, 3)
AETH_FLUX_INST(double, 4)
#undef AETH_FLUX_INST

}  // namespace aeth
