// Static SOX for periodic solids, FP64 complex (kpoint.cu).
#pragma once
#include "internal.h"

namespace sox {
struct KpointPlan {
  int nk = 1;        // k-points of the mesh
  int nv = 1;        // v values per chunk of B and C
  size_t fixed_bytes = 0, bytes = 0;
};
KpointPlan kpoint_plan(sox_handle h, int n, int N, int T, int S, const int nk[3]);
// Sigma^k(tau) for every spin, k and tau; G, X, U1, U2, Sigma are device arrays of
// interleaved complex doubles in the library layout.  U1 == U2 for bare SOX.
Status kpoint_sigma_f64(sox_handle h, const sox_problem *p, const double *G, const double *X, const double *U1,
                        const double *U2, double *Sigma, Arena &ar, cudaStream_t s);
// Dynamically screened SOSEX for solids: Sigma += Sigma_d with W_d^{q}(i Omega_m)
// [n_q][n_omega][N][N] in the first interaction slot and the bare V^q in the second;
// T_fwd [n_omega][n_tau], T_inv [n_tau][n_omega] the caller's transform pair.  All
// device arrays of interleaved complex doubles; Sigma already holds SOX(v, v).
size_t kpoint_dynamic_bytes(sox_handle h, int n, int N, int T, int n_omega, const int nk[3], int *ct_out);
Status kpoint_dynamic_add_f64(sox_handle h, const sox_problem *p, int n_omega, const double *G, const double *X,
                              const double *V, const double *Wd, const double *T_fwd, const double *T_inv,
                              double *Sigma, Arena &ar, cudaStream_t s);
// RPA screened interaction W_d^q(i Omega_o) = (1 - V^q Pi^q)^-1 V^q - V^q on the transform's
// frequencies for every transfer q (molecules: the mesh 1x1x1, real data, real W_d
// [n_omega][N][N]; solids: complex W_d [n_q][n_omega][N][N]); device inputs in the
// library layouts, T_fwd [n_omega][n_tau] complex.  Synchronises s (reads the singular flag).
size_t w_dynamic_bytes(const sox_problem *p, int n_omega);
Status w_dynamic(sox_handle h, const sox_problem *p, int n_omega, const double *G, const double *X, const double *V,
                 const double *T_fwd, double *Wd, Arena &ar, cudaStream_t s);
}  // namespace sox
