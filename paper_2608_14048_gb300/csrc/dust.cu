// Multifluid dust (filled in below).
#include "runtime.hpp"
namespace aeth {
template <typename R, bool P64>
aeth_status step_dust(aeth_ctx* c) { return fail(c, AETH_ERR_UNSUPPORTED, "dust path not built"); }
template aeth_status step_dust<float, false>(aeth_ctx*);
template aeth_status step_dust<float, true>(aeth_ctx*);
template aeth_status step_dust<double, false>(aeth_ctx*);
}  // namespace aeth
extern "C" aeth_status aeth_load_mlp(aeth_ctx* c, const float*, size_t) {
  return c ? aeth::fail(c, AETH_ERR_UNSUPPORTED, "learned flux not built") : AETH_ERR_ARG;
}
