// Learned Riemann flux (filled in below).
#include "runtime.hpp"
extern "C" aeth_status aeth_load_mlp(aeth_ctx* c, const float*, size_t) {
  return c ? aeth::fail(c, AETH_ERR_UNSUPPORTED, "learned flux not built") : AETH_ERR_ARG;
}
