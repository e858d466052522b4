// Dynamically screened SOSEX for molecules (Sec. II C, Eq. GG and the steps after
// it), FP64 on CUDA cores.  The screened part W_d = W - v sits in slot U(1); the
// static part SOX(v, v) comes from the static path.
//
// For every v (outer loop, as the paper moves it outside for memory):
//   GG[j][Q][u]   = G_uQ(tau_j) G_Qv(-tau_j)         G_uQ = GWt_j[Q][u], G_Qv(-tau_j) = -GR_{T-1-j}[Q][v]
//   GGw[m]        = sum_j T_fwd[m][j] GG[j]           (complex, re/im interleaved)
//   Aw[m][P][u]   = sum_Q W_d[m][P][Q] GGw[m][Q][u]   (real W_d acts on re and im alike)
//   A[i][v][P][u] = Re sum_m T_inv[i][m] Aw[m][P][u]
// then B_v[P][R] = sum_u A[i][v][P][u] X[R][u], C_v[P][R] = sum_w GWt_i[P][w] U[R][v][w] and
// D = sum_v B_v o C_v are exactly the fused static kernel with X in the G_Rq slot, and
// Sigma_d = -X^T D^T X is added to Sigma.
#include <algorithm>

#include "dynamic.h"

namespace sox {
namespace {

// GG[j][Q][u] = GWt[j][Q][u] * (-GR[T-1-j][Q][v])
__global__ void k_gg(const double *GWt, const double *GR, int T, int N, int n, int v, double *GG) {
  const long long Nn = (long long)N * n, total = Nn * T;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / Nn);
    const long long r = e % Nn;
    const int Q = (int)(r / n);
    GG[e] = -GWt[e] * GR[(long long)(T - 1 - j) * Nn + (long long)Q * n + v];
  }
}

int grid1(long long total) { return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 65535 * 8)); }

}  // namespace

size_t dynamic_bytes(int n, int N, int T, int n_omega) {
  const size_t Nn = (size_t)N * n;
  return 8 * ((size_t)N * n * n /*Um*/ + (size_t)N * n * n /*pairs*/ + 2 * (size_t)T * Nn /*GR, GWt*/ +
              (size_t)T * Nn /*GG*/ + 4 * (size_t)n_omega * Nn /*GGw, Aw*/ + (size_t)T * n * Nn /*A*/ +
              (size_t)T * N * N /*D*/ + (size_t)T * Nn /*T*/) +
         64 * 1024;
}

Status dynamic_sigma_add_f64(sox_handle h, int n, int N, int T, int S, int n_omega, const double *G, const double *X,
                             const double *V, const double *Wd, const double *Tf, const double *Ti, double *Sigma,
                             Arena &ar, cudaStream_t s) {
  const long long nn = (long long)n * n, Nn = (long long)N * n, NN = (long long)N * N;
  double *Um = ar.take<double>((size_t)N * nn), *Y = ar.take<double>((size_t)N * nn);
  double *GR = ar.take<double>((size_t)T * Nn), *GWt = ar.take<double>((size_t)T * Nn);
  double *GG = ar.take<double>((size_t)T * Nn);
  double *GGw = ar.take<double>((size_t)2 * n_omega * Nn), *Aw = ar.take<double>((size_t)2 * n_omega * Nn);
  double *A = ar.take<double>((size_t)T * n * Nn);
  double *D = ar.take<double>((size_t)T * NN), *Tm = ar.take<double>((size_t)T * Nn);
  if (!Tm) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  ProfScope ps(h, "sosex_dynamic_f64", s, 0);
  long long launches = 0;
  int v_lo = 0, v_hi = n;   // the handle's v range (sox_set_v_range)
  v_range(h, n, &v_lo, &v_hi);
  // U[P][q][s] = sum_Q V[P][Q] X[Q][q] X[Q][s]
  launch_pair_products_f64(X, Y, N, n, s);
  GemmF64 m;
  m.M = N; m.Nc = (int)nn; m.K = N;
  m.A = V; m.ai = N; m.ak = 1;
  m.B = Y; m.bk = nn; m.bj = 1;
  m.C = Um; m.ci = nn; m.cj = 1;
  launch_gemm_f64(m, s);
  launches += 2;
  for (int sp = 0; sp < S; ++sp) {
    const double *Gs = G + (long long)sp * T * nn;
    GemmF64 g;  // GR[j][R][q] = sum_u X[R][u] G_j[u][q]
    g.M = N; g.Nc = n; g.K = n; g.batch = T;
    g.A = X; g.ai = n; g.ak = 1;
    g.B = Gs; g.sB = nn; g.bk = n; g.bj = 1;
    g.C = GR; g.sC = Nn; g.ci = n; g.cj = 1;
    launch_gemm_f64(g, s);
    GemmF64 gw = g;  // GWt[j][P][w] = sum_p X[P][p] G_j[w][p]
    gw.bk = 1; gw.bj = n; gw.C = GWt;
    launch_gemm_f64(gw, s);
    launches += 2;
    for (int v = v_lo; v < v_hi; ++v) {
      k_gg<<<grid1((long long)T * Nn), 256, 0, s>>>(GWt, GR, T, N, n, v, GG);
      for (int c = 0; c < 2; ++c) {  // GGw[m][(Q,u)][c] = sum_j {Re, Im} T_fwd[m][j] GG[j][(Q,u)]
        GemmF64 f;
        f.M = n_omega; f.Nc = (int)Nn; f.K = T;
        f.A = Tf + c; f.ai = 2LL * T; f.ak = 2;
        f.B = GG; f.bk = Nn; f.bj = 1;
        f.C = GGw + c; f.ci = 2 * Nn; f.cj = 2;
        launch_gemm_f64(f, s);
      }
      GemmF64 w;  // Aw[m][P][(u,c)] = sum_Q Wd[m][P][Q] GGw[m][Q][(u,c)]
      w.M = N; w.Nc = 2 * n; w.K = N; w.batch = n_omega;
      w.A = Wd; w.sA = NN; w.ai = N; w.ak = 1;
      w.B = GGw; w.sB = 2 * Nn; w.bk = 2LL * n; w.bj = 1;
      w.C = Aw; w.sC = 2 * Nn; w.ci = 2LL * n; w.cj = 1;
      launch_gemm_f64(w, s);
      // A[i][v][(P,u)] = sum_m Re T_inv[i][m] Re Aw[m] - Im T_inv[i][m] Im Aw[m]
      for (int c = 0; c < 2; ++c) {
        GemmF64 iv;
        iv.M = T; iv.Nc = (int)Nn; iv.K = n_omega;
        iv.A = Ti + c; iv.ai = 2LL * n_omega; iv.ak = 2;
        iv.B = Aw + c; iv.bk = 2 * Nn; iv.bj = 2;
        iv.C = A + (long long)v * Nn; iv.ci = (long long)n * Nn; iv.cj = 1;
        iv.alpha = c == 0 ? 1.0 : -1.0;
        iv.beta = c == 0 ? 0.0 : 1.0;
        launch_gemm_f64(iv, s);
      }
      launches += 6;
    }
    // D[i] = sum_v (A[i][v] X^T) o (GWt_i U_v^T): the fused kernel with X in the G_Rq slot
    launch_sox_bcd_f64(A, (long long)n * Nn, X, 0, GWt, Nn, Um, D, NN, n, N, T, s, v_lo, v_hi);
    GemmF64 t;  // T[i][R][r] = sum_P D[i][P][R] X[P][r]
    t.M = N; t.Nc = n; t.K = N; t.batch = T;
    t.A = D; t.sA = NN; t.ai = 1; t.ak = N;
    t.B = X; t.bk = n; t.bj = 1;
    t.C = Tm; t.sC = Nn; t.ci = n; t.cj = 1;
    launch_gemm_f64(t, s);
    GemmF64 b;  // Sigma[i][t][r] += -sum_R X[R][t] T[i][R][r]
    b.M = n; b.Nc = n; b.K = N; b.batch = T;
    b.A = X; b.ai = 1; b.ak = n;
    b.B = Tm; b.sB = Nn; b.bk = n; b.bj = 1;
    b.C = Sigma + (long long)sp * T * nn; b.sC = nn; b.ci = n; b.cj = 1;
    b.alpha = -1.0; b.beta = 1.0;
    launch_gemm_f64(b, s);
    launches += 3;
  }
  h->launches += launches;
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

}  // namespace sox
