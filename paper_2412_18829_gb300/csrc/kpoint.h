// Static SOX for periodic solids, FP64 complex (kpoint.cu).
#pragma once
#include "internal.h"

namespace sox {
struct KpointPlan {
  int nk = 1;        // k-points of the mesh
  int nv = 1;        // v values per chunk of B and C
  size_t fixed_bytes = 0, bytes = 0;
};
KpointPlan kpoint_plan(int n, int N, int T, int S, const int nk[3]);
// Sigma^k(tau) for every spin, k and tau; G, X, U1, U2, Sigma are device arrays of
// interleaved complex doubles in the library layout.  U1 == U2 for bare SOX.
Status kpoint_sigma_f64(sox_handle h, const sox_problem *p, const double *G, const double *X, const double *U1,
                        const double *U2, double *Sigma, Arena &ar, cudaStream_t s);
}  // namespace sox
