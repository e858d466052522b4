#include "tc_path.h"

namespace sox {
size_t tc_sigma_bytes(sox_handle, int, int, int, int, bool) { return 0; }
Status tc_sigma(sox_handle, int, int, int, int, const double *, const double *, const double *,
                const double *, double *, Arena &, cudaStream_t) {
  return {SOX_ERR_UNSUPPORTED, "tensor-core path not built"};
}
void tc_release(sox_handle) {}
}  // namespace sox
