// Reverse-mode adjoint of Phi_SOX with respect to X and V (adjoint.cu).
#pragma once
#include "internal.h"

namespace sox {
// Workspace bytes of phi_adjoint_xv_f64; *chunk receives the tau points per pass.
size_t adjoint_bytes(sox_handle h, int n, int N, int T, int S, int *chunk);
// dX[P][p] = sum_s dphi[s] dPhi_s/dX[P][p],  dV[P][Q] = sum_s dphi[s] dPhi_s/dV[P][Q]  (bare SOX,
// FP64).  G, X, V, w, dphi device pointers; dX / dV may be NULL.
Status phi_adjoint_xv_f64(sox_handle h, int n, int N, int T, int S, const double *G, const double *X,
                          const double *V, const double *w, const double *dphi, double *dX, double *dV,
                          Arena &ar, cudaStream_t s);
// The same in split precision (adjoint_tc.cu): every N x N x n contraction of the reverse
// pass on the tensor cores in FP16 pairs with FP32 accumulation; FP64 projections.
size_t adjoint_tc_bytes(sox_handle h, int n, int N, int T, int S);
Status phi_adjoint_xv_tc(sox_handle h, int n, int N, int T, int S, const double *G, const double *X,
                         const double *V, const double *w, const double *dphi, double *dX, double *dV,
                         Arena &ar, cudaStream_t s);
}  // namespace sox
