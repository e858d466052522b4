// Dynamically screened SOSEX for molecules (dynamic.cu).
#pragma once
#include "internal.h"

namespace sox {
size_t dynamic_bytes(int n, int N, int T, int n_omega);
// Sigma[s][0][i] += Sigma_d(tau_i) for every spin (FP64; Sigma already holds SOX(v, v)).
// Wd [n_omega][N][N] real; Tf [n_omega][T] and Ti [T][n_omega] complex interleaved.
Status dynamic_sigma_add_f64(sox_handle h, int n, int N, int T, int S, int n_omega, const double *G, const double *X,
                             const double *V, const double *Wd, const double *Tf, const double *Ti, double *Sigma,
                             Arena &ar, cudaStream_t s);
// The same in split precision (dynamic_tc.cu): the transforms and the W_d product as
// FP16-pair GEMMs on the tensor cores, then the fused B/C/D kernel with X in the G_Rq slot.
size_t dynamic_tc_bytes(sox_handle h, int n, int N, int T, int S, int n_omega);
Status dynamic_sigma_add_tc(sox_handle h, int n, int N, int T, int S, int n_omega, const double *G, const double *X,
                            const double *V, const double *Wd, const double *Tf, const double *Ti, double *Sigma,
                            Arena &ar, cudaStream_t s);
}  // namespace sox
