// tcgen05 (sm_103a) tensor-core kernels for the SPSVM_BF16X3 form.
#include "internal.h"
#include "gram.h"

namespace spsvm {

bool tc_available() { return false; }

int launch_kernel_block_tc(const spsvm_points*, const int64_t*, int32_t, float, spsvm_kmat*,
                           int64_t, cudaStream_t) {
  return set_error(SPSVM_ERR_ARG, "BF16X3 kernel block not built");
}

int64_t score_tc_tiles(int64_t n) { return ceil_div(n, (int64_t)128); }

int launch_score_tc(const spsvm_points*, const float*, const float*, const int64_t*, int32_t,
                    float, double2*, int64_t, cudaStream_t) {
  return set_error(SPSVM_ERR_ARG, "BF16X3 score not built");
}

int64_t gram_tc_splits(int64_t m, int64_t ns_max) { (void)m; (void)ns_max; return 1; }

int launch_gram_tc(const spsvm_kmat*, const int64_t*, int64_t, int64_t, double*, int64_t, int64_t,
                   cudaStream_t) {
  return set_error(SPSVM_ERR_ARG, "BF16X3 gram not built");
}

}  // namespace spsvm
