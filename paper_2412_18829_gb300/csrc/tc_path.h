// Mixed-precision (tcgen05 tensor-core) path of the THC-SOX chain.
#pragma once
#include "internal.h"

namespace sox {
size_t tc_sigma_bytes(sox_handle h, int n, int N, int T, int S, bool two_slots);
Status tc_sigma(sox_handle h, int n, int N, int T, int S, const double *G, const double *X,
                const double *U1, const double *U2, double *Sigma, Arena &ar, cudaStream_t s);
void tc_release(sox_handle h);
}  // namespace sox
