// Fused stage kernel (filled in below).
#include "runtime.hpp"
namespace aeth {
bool fused_supported(const aeth_ctx*) { return false; }
template <typename R, bool P64>
aeth_status step_fused(aeth_ctx* c) { return fail(c, AETH_ERR_UNSUPPORTED, "fused path not built"); }
template aeth_status step_fused<float, false>(aeth_ctx*);
template aeth_status step_fused<float, true>(aeth_ctx*);
template aeth_status step_fused<double, false>(aeth_ctx*);
}  // namespace aeth
