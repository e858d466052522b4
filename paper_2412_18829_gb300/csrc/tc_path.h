// Mixed-precision (tcgen05 tensor-core) path of the THC-SOX chain.
#pragma once
#include "internal.h"

namespace sox {
size_t tc_sigma_bytes(sox_handle h, int n, int N, int T, int S, bool two_slots);
Status tc_sigma(sox_handle h, int n, int N, int T, int S, const double *G, const double *X,
                const double *U1, const double *U2, double *Sigma, Arena &ar, cudaStream_t s);
void tc_release(sox_handle h);
// The uneven batch of bare-SOX molecules: per-instance chains, one persistent fused launch per
// tau chunk over every instance's tiles.  Arrays of `count` shapes; U1 = U2 = V per instance.
size_t tc_sigma_batch_bytes(sox_handle h, int count, const int *n, const int *N, const int *T, const int *S);
Status tc_sigma_batch(sox_handle h, int count, const int *n, const int *N, const int *T, const int *S,
                      const double *const *G, const double *const *X, const double *const *V, double *const *Sigma,
                      Arena &ar, cudaStream_t s);
}  // namespace sox
