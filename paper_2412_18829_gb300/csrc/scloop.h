// The self-consistent loop's device steps (scloop.cu).
#pragma once
#include "internal.h"

namespace sox {
// G_iw[s][w] = [(i w + mu) 1 - F[s] - Sigma_iw[s][w]]^-1 for every spin and frequency (complex
// Gauss-Jordan with partial pivoting, one block per system); Sigma_iw may be NULL.  Device
// pointers; synchronises s to report a singular system.
size_t dyson_bytes(int n, int n_w, int n_spin);
Status dyson(sox_handle h, int n, int n_w, int n_spin, const double *omegas, double mu, const double *F,
             const double *Sigma_iw, double *G_iw, Arena &ar, cudaStream_t s);
// tails[s] = {1, F - mu, (F - mu)^2 - (Sigma(tau_{T-1}) + Sigma(tau_0))}, real [n_spin][3][n][n]
void launch_green_tails(const double *F, double mu, const double *Sigma_tau, int n, int T, int n_spin, double *tails,
                        cudaStream_t s);
void launch_iw_to_tau(const double *G_iw, const double *omegas, int n_w, const double *tails, const double *tau,
                      int n_t, int n, int n_spin, double beta, double *G_tau, cudaStream_t s);
void launch_tau_to_iw(const double *Tw, const double *F_tau, int n_w, int T, int n, int n_spin, double *F_iw,
                      cudaStream_t s);
// count[0] += sum_s Tr gamma^s with gamma = -G(beta^-)^T
void launch_trace_gamma(const double *G_iw, const double *omegas, int n_w, const double *tails, int n, int n_spin,
                        double beta, double *count, cudaStream_t s);
// d: N + n_spin N n doubles of scratch; Gam: n_spin N N
void launch_sigma_hf(const double *X, const double *V, const double *gamma, int N, int n, int n_spin, double *d,
                     double *Gam, double *S, cudaStream_t s);
// out[0] += E_inf, out[1] += E_dyn (out zeroed by the caller)
void launch_energies(const double *H0, const double *Shf, const double *gamma, const double *Sigma_tau,
                     const double *G_tau, const double *w, int n, int T, int n_spin, double *out, cudaStream_t s);
// gamma[s][p][q] = -G[s][n_tau-1][q][p]  (gamma = G(0^-) = -G(beta^-), read transposed)
void launch_gamma_from_tau(const double *G_tau, int n, int T, int n_spin, double *gamma, cudaStream_t s);
void launch_mix(double *G, const double *Gnew, long long count, double a, unsigned long long *change, cudaStream_t s);
}  // namespace sox
