// Shared declarations of the Gram-matrix (masked SYRK) launchers.
#pragma once
#include "internal.h"

namespace spsvm {

// Points per FP32 partial sum before promotion to FP64.
constexpr int64_t GRAM_SLICE = 8192;

int64_t gram_simt_splits(int64_t m, int64_t ns_max);
int launch_gram_simt(const spsvm_kmat* Kc, const int64_t* ns_dev, int64_t ns_max, int64_t m,
                     double* part, int64_t ldp, int64_t splits, cudaStream_t s);

// kjj: the symmetric K_JJ (FP64, row pitch ldk) if the caller keeps one, else
// NULL (gathered from K into the scratch behind the partial sums).
int gram_impl(const spsvm_kmat* Kc, const int64_t* ns_dev, int64_t ns_max, const spsvm_kmat* K,
              const int64_t* J, double lambda, int32_t precision, double* H, int64_t ldh,
              void* scratch, size_t scratch_bytes, cudaStream_t s, double ns_work,
              const double* kjj, int64_t ldk);

// Scratch of the partial sums alone (with a caller-kept K_JJ).
size_t gram_part_bytes(int64_t m, int64_t ns);

// K_JJ entries in the rows and columns row0 .. m-1 (see gram_simt.cu).
int kjj_fill(const spsvm_kmat* K, const int64_t* J, int64_t m, int64_t row0, double* kjj,
             int64_t ldk, cudaStream_t s);

int64_t gram_tc_splits(int64_t m, int64_t ns_max);
int launch_gram_tc(const spsvm_kmat* Kc, const int64_t* ns_dev, int64_t ns_max, int64_t m,
                   double* part, int64_t ldp, int64_t splits, cudaStream_t s);

}  // namespace spsvm
