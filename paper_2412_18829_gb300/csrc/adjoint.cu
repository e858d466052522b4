// Adjoint of the Luttinger-Ward functional of bare SOX with respect to X and V
// (FP64), by reverse mode through the THC chain of Sec. II C with the
// intermediates recomputed per tau chunk instead of stored.
//
// Forward (one spin, tau_j; X[P][p], U = V mixed as Um[P][q][s]):
//   GR = X G_j, GWt = X G_j^T, A[v][P][q] = sum_s Gm_j[s][v] Um[P][q][s]
//   B_v[P][R] = sum_q A[v][P][q] GR[R][q],  C_v[P][R] = sum_w GWt[P][w] Um[R][v][w]
//   D = sum_v B_v o C_v,  E = X Gm_j X^T  (= G^PR(-tau_j))
//   Phi = 1/4 sum_j w_j Tr[Sigma_j G(-tau_j)] = -1/4 sum_j w_j sum_PR D[P][R] E[P][R]
// Reverse, with c_j = -w_j dphi / 4:
//   Dbar = c_j E,  Ebar = c_j D
//   Bbar_v = Dbar o C_v,  Cbar_v = Dbar o B_v
//   Abar[v][P][q]  = sum_R Bbar_v[P][R] GR[R][q]
//   GRbar[R][q]    = sum_v sum_P Bbar_v[P][R] A[v][P][q]
//   GWtbar[P][w]   = sum_v sum_R Cbar_v[P][R] Um[R][v][w]
//   U2bar[R][v][w] = sum_j sum_P Cbar_v[P][R] GWt[P][w]
//   U1bar[P][q][s] = sum_j sum_v Abar[v][P][q] Gm_j[s][v]
//   Xbar += GRbar G_j^T + GWtbar G_j + Ebar X Gm_j^T + Ebar^T X Gm_j
//   Vbar  = (U1bar + U2bar) Y^T,   Y[Q][(q,s)] = X[Q][q] X[Q][s]
//   Xbar[Q][q] += sum_s (Z[Q][q][s] + Z[Q][s][q]) X[Q][s],   Z = V^T (U1bar + U2bar)
// (V enters both mixed tensors of bare SOX; V^T = V is not assumed.)
#include <algorithm>

#include "adjoint.h"

namespace sox {
namespace {

constexpr int TM = 64, TK = 16, NT = 256;

// One (P, R) tile of 64 x 64 per block: recompute B_v, C_v for every v and write
// Bbar[v][j][P][R] = Dbar[j][P][R] C_v and Cbar[v][j][P][R] = Dbar[j][P][R] B_v.
__global__ void __launch_bounds__(NT) k_bcd_adjoint_f64(const double *A, long long sA, const double *GR,
                                                       long long sGR, const double *GWt, long long sGW,
                                                       const double *Um, const double *Dbar, long long sD,
                                                       double *Bbar, double *Cbar, int n, int N, int cj) {
  __shared__ double s_a[TK][TM + 1];
  __shared__ double s_gr[TK][TM + 1];
  __shared__ double s_gw[TK][TM + 1];
  __shared__ double s_u[TK][TM + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int P0 = blockIdx.y * TM, R0 = blockIdx.x * TM;
  const int j = blockIdx.z;
  const double *Ab = A + j * sA, *GRb = GR + j * sGR, *GWb = GWt + j * sGW;
  const long long nn = (long long)n * n, NN = (long long)N * N;
  double db[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int P = P0 + ty + 16 * i, R = R0 + tx + 16 * k;
      db[i][k] = (P < N && R < N) ? Dbar[j * sD + (long long)P * N + R] : 0.0;
    }
  auto load = [&](double(*s)[TM + 1], const double *base, long long rs, int r0, int k0) {
#pragma unroll
    for (int it = 0; it < (TM * TK) / NT; ++it) {
      const int e = tid + it * NT;
      const int r = e / TK, k = e % TK;
      const int gr = r0 + r, gk = k0 + k;
      s[k][r] = (gr < N && gk < n) ? base[gr * rs + gk] : 0.0;
    }
  };
  for (int v = 0; v < n; ++v) {
    double bacc[4][4] = {}, cacc[4][4] = {};
    const double *Av = Ab + (long long)v * N * n;
    const double *Uv = Um + (long long)v * n;
    for (int k0 = 0; k0 < n; k0 += TK) {
      load(s_a, Av, n, P0, k0);
      load(s_gr, GRb, n, R0, k0);
      load(s_gw, GWb, n, P0, k0);
      load(s_u, Uv, nn, R0, k0);
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < TK; ++kk) {
        double a[4], gr[4], gw[4], u[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          a[i] = s_a[kk][ty + 16 * i];
          gw[i] = s_gw[kk][ty + 16 * i];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          gr[k] = s_gr[kk][tx + 16 * k];
          u[k] = s_u[kk][tx + 16 * k];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            bacc[i][k] = fma(a[i], gr[k], bacc[i][k]);
            cacc[i][k] = fma(gw[i], u[k], cacc[i][k]);
          }
      }
      __syncthreads();
    }
    const long long base = ((long long)v * cj + j) * NN;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int P = P0 + ty + 16 * i;
      if (P >= N) continue;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int R = R0 + tx + 16 * k;
        if (R >= N) continue;
        Bbar[base + (long long)P * N + R] = db[i][k] * cacc[i][k];
        Cbar[base + (long long)P * N + R] = db[i][k] * bacc[i][k];
      }
    }
  }
}

// out[b] = scale[b] * in[b]  (per-batch scaling of N x N blocks; scale = -w_j dphi / 4)
__global__ void k_scale_blocks(const double *in, double *out, long long blk, int count, const double *w,
                               const double *dphi, int t0) {
  const long long total = blk * count;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / blk);
    out[e] = -0.25 * w[t0 + j] * dphi[0] * in[e];
  }
}

// dst[i] += sum_j src[j][i]
__global__ void k_sum_batches(const double *src, long long len, int count, double *dst) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < count; ++j) acc += src[(long long)j * len + e];
    dst[e] += acc;
  }
}

// Xbar[Q][q] += sum_s (Z[Q][q][s] + Z[Q][s][q]) X[Q][s]
__global__ void k_pair_adjoint(const double *Z, const double *X, int N, int n, double *Xbar) {
  const long long total = (long long)N * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int Q = (int)(e / n), q = (int)(e % n);
    const double *z = Z + (long long)Q * n * n;
    const double *x = X + (long long)Q * n;
    double acc = 0.0;
    for (int s = 0; s < n; ++s) acc = fma(z[(long long)q * n + s] + z[(long long)s * n + q], x[s], acc);
    Xbar[e] += acc;
  }
}

int grid1(long long total) { return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 65535 * 8)); }

}  // namespace

size_t adjoint_bytes(sox_handle h, int n, int N, int T, int S, int *chunk) {
  const size_t nn = (size_t)n * n, Nn2 = (size_t)N * nn, NN = (size_t)N * N, Nn = (size_t)N * n;
  const size_t fixed = 8 * (2 * Nn2 /*Um, Y*/ + 2 * Nn2 /*U1bar, U2bar*/ + Nn2 /*Z*/ + Nn + NN) + 4096 * 16;
  const size_t per_j = 8 * (2 * Nn2 /*A, Abar*/ + 4 * Nn /*GR, GWt, GRbar, GWtbar*/ + 3 * NN /*D, E, Dbar/Ebar*/ +
                            2 * (size_t)n * NN /*Bbar, Cbar*/ + 3 * Nn /*Xbar parts, M1, M2*/ + Nn) + 4096;
  const size_t budget = chunk_budget(h, size_t(16) << 30);
  long long c = budget > fixed ? (long long)((budget - fixed) / per_j) : 1;
  c = std::max<long long>(1, std::min<long long>(c, T));
  if (chunk) *chunk = (int)c;
  (void)S;
  return fixed + per_j * c + 4096 * 32;
}

Status phi_adjoint_xv_f64(sox_handle h, int n, int N, int T, int S, const double *G, const double *X,
                          const double *V, const double *w, const double *dphi, double *dX, double *dV,
                          Arena &ar, cudaStream_t s) {
  int c = 1;
  adjoint_bytes(h, n, N, T, S, &c);
  const long long nn = (long long)n * n, Nn2 = (long long)N * nn, NN = (long long)N * N, Nn = (long long)N * n;
  double *Um = ar.take<double>(Nn2), *Y = ar.take<double>(Nn2);
  double *U1bar = ar.take<double>(Nn2), *U2bar = ar.take<double>(Nn2), *Z = ar.take<double>(Nn2);
  double *Xbar = ar.take<double>(Nn), *Vbar = ar.take<double>(NN);
  double *A = ar.take<double>((size_t)c * Nn2), *Abar = ar.take<double>((size_t)c * Nn2);
  double *GR = ar.take<double>((size_t)c * Nn), *GWt = ar.take<double>((size_t)c * Nn);
  double *GRbar = ar.take<double>((size_t)c * Nn), *GWtbar = ar.take<double>((size_t)c * Nn);
  double *D = ar.take<double>((size_t)c * NN), *E = ar.take<double>((size_t)c * NN);
  double *Sc = ar.take<double>((size_t)c * NN);
  double *Bbar = ar.take<double>((size_t)c * n * NN), *Cbar = ar.take<double>((size_t)c * n * NN);
  double *Xpart = ar.take<double>((size_t)c * Nn), *M1 = ar.take<double>((size_t)c * Nn);
  double *M2 = ar.take<double>((size_t)c * Nn);
  if (!M2) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};

  ProfScope ps(h, "phi_adjoint_f64", s, 0);
  long long launches = 0;
  int v_lo = 0, v_hi = n;   // the handle's v range (sox_set_v_range): Phi's v sum runs over [v_lo, v_hi)
  v_range(h, n, &v_lo, &v_hi);
  SOX_CUDA_TRY(cudaMemsetAsync(U1bar, 0, 8 * Nn2, s));
  SOX_CUDA_TRY(cudaMemsetAsync(U2bar, 0, 8 * Nn2, s));
  SOX_CUDA_TRY(cudaMemsetAsync(Xbar, 0, 8 * Nn, s));
  // Um[P][q][s] = sum_Q V[P][Q] X[Q][q] X[Q][s]
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
    for (int t0 = 0; t0 < T; t0 += c) {
      const int cc = std::min(c, T - t0);
      // forward recomputation: GR, GWt, A, D, E
      GemmF64 g;
      g.M = N; g.Nc = n; g.K = n; g.batch = cc;
      g.A = X; g.ai = n; g.ak = 1;
      g.B = Gs + (long long)t0 * nn; g.sB = nn; g.bk = n; g.bj = 1;
      g.C = GR; g.sC = Nn; g.ci = n; g.cj = 1;
      launch_gemm_f64(g, s);
      GemmF64 gw = g;
      gw.bk = 1; gw.bj = n;
      gw.C = GWt;
      launch_gemm_f64(gw, s);
      GemmF64 a;  // A[j][v][(P,q)] = -sum_s G(tau_{T-1-j})[s][v] Um[(P,q)][s]
      a.M = n; a.Nc = N * n; a.K = n; a.batch = cc;
      a.A = Gs + (long long)(T - 1 - t0) * nn; a.sA = -nn; a.ai = 1; a.ak = n;
      a.B = Um; a.bk = 1; a.bj = n;
      a.C = A; a.sC = Nn2; a.ci = Nn; a.cj = 1;
      a.alpha = -1.0;
      launch_gemm_f64(a, s);
      launch_sox_bcd_f64(A, Nn2, GR, Nn, GWt, Nn, Um, D, NN, n, N, cc, s, v_lo, v_hi);
      // E[j] = X Gm_j X^T = -X G_{T-1-j} X^T : M1 = -X G_{T-1-j}, E = M1 X^T
      GemmF64 e1;
      e1.M = N; e1.Nc = n; e1.K = n; e1.batch = cc;
      e1.A = X; e1.ai = n; e1.ak = 1;
      e1.B = Gs + (long long)(T - 1 - t0) * nn; e1.sB = -nn; e1.bk = n; e1.bj = 1;
      e1.C = M1; e1.sC = Nn; e1.ci = n; e1.cj = 1;
      e1.alpha = -1.0;
      launch_gemm_f64(e1, s);
      GemmF64 e2;
      e2.M = N; e2.Nc = N; e2.K = n; e2.batch = cc;
      e2.A = M1; e2.sA = Nn; e2.ai = n; e2.ak = 1;
      e2.B = X; e2.bk = 1; e2.bj = n;
      e2.C = E; e2.sC = NN; e2.ci = N; e2.cj = 1;
      launch_gemm_f64(e2, s);
      launches += 6;
      // Dbar = c_j E (into Sc), then Bbar, Cbar
      k_scale_blocks<<<grid1(NN * cc), 256, 0, s>>>(E, Sc, NN, cc, w, dphi + sp, t0);
      {
        dim3 grid((N + TM - 1) / TM, (N + TM - 1) / TM, cc);
        k_bcd_adjoint_f64<<<grid, NT, 0, s>>>(A, Nn2, GR, Nn, GWt, Nn, Um, Sc, NN, Bbar, Cbar, n, N, cc);
      }
      launches += 2;
      SOX_CUDA_TRY(cudaMemsetAsync(GRbar, 0, 8 * Nn * cc, s));
      SOX_CUDA_TRY(cudaMemsetAsync(GWtbar, 0, 8 * Nn * cc, s));
      for (int v = v_lo; v < v_hi; ++v) {
        const double *Bb = Bbar + (long long)v * cc * NN;   // [j][P][R]
        const double *Cb = Cbar + (long long)v * cc * NN;
        GemmF64 ab;  // Abar[j][v][P][q] = sum_R Bbar_v[j][P][R] GR[j][R][q]
        ab.M = N; ab.Nc = n; ab.K = N; ab.batch = cc;
        ab.A = Bb; ab.sA = NN; ab.ai = N; ab.ak = 1;
        ab.B = GR; ab.sB = Nn; ab.bk = n; ab.bj = 1;
        ab.C = Abar + (long long)v * Nn; ab.sC = Nn2; ab.ci = n; ab.cj = 1;
        launch_gemm_f64(ab, s);
        GemmF64 grb;  // GRbar[j][R][q] += sum_P Bbar_v[j][P][R] A[j][v][P][q]
        grb.M = N; grb.Nc = n; grb.K = N; grb.batch = cc;
        grb.A = Bb; grb.sA = NN; grb.ai = 1; grb.ak = N;
        grb.B = A + (long long)v * Nn; grb.sB = Nn2; grb.bk = n; grb.bj = 1;
        grb.C = GRbar; grb.sC = Nn; grb.ci = n; grb.cj = 1;
        grb.beta = 1.0;
        launch_gemm_f64(grb, s);
        GemmF64 gwb;  // GWtbar[j][P][w] += sum_R Cbar_v[j][P][R] Um[R][v][w]
        gwb.M = N; gwb.Nc = n; gwb.K = N; gwb.batch = cc;
        gwb.A = Cb; gwb.sA = NN; gwb.ai = N; gwb.ak = 1;
        gwb.B = Um + (long long)v * n; gwb.bk = nn; gwb.bj = 1;
        gwb.C = GWtbar; gwb.sC = Nn; gwb.ci = n; gwb.cj = 1;
        gwb.beta = 1.0;
        launch_gemm_f64(gwb, s);
        GemmF64 u2;  // U2bar[R][v][w] += sum_{(j,P)} Cbar_v[j][P][R] GWt[j][P][w]
        u2.M = N; u2.Nc = n; u2.K = N * cc;
        u2.A = Cb; u2.ai = 1; u2.ak = N;
        u2.B = GWt; u2.bk = n; u2.bj = 1;
        u2.C = U2bar + (long long)v * n; u2.ci = nn; u2.cj = 1;
        u2.beta = 1.0;
        launch_gemm_f64(u2, s);
        launches += 4;
      }
      // U1bar[(P,q)][s] += sum_v Abar[j][v][(P,q)] Gm_j[s][v]   (one launch per j: shared output)
      for (int j = 0; j < cc; ++j) {
        GemmF64 u1;   // K = v over the handle's v range
        u1.M = N * n; u1.Nc = n; u1.K = v_hi - v_lo;
        u1.A = Abar + (long long)j * Nn2 + (long long)v_lo * Nn; u1.ai = 1; u1.ak = Nn;
        u1.B = Gs + (long long)(T - 1 - (t0 + j)) * nn + v_lo; u1.bk = 1; u1.bj = n;
        u1.C = U1bar; u1.ci = n; u1.cj = 1;
        u1.alpha = -1.0; u1.beta = 1.0;
        launch_gemm_f64(u1, s);
        ++launches;
      }
      // Xbar parts per j: GRbar G_j^T + GWtbar G_j + Ebar X Gm_j^T + Ebar^T X Gm_j, Ebar = c_j D
      k_scale_blocks<<<grid1(NN * cc), 256, 0, s>>>(D, Sc, NN, cc, w, dphi + sp, t0);
      GemmF64 x1;  // Xpart[j][R][u] = sum_q GRbar[j][R][q] G_j[u][q]
      x1.M = N; x1.Nc = n; x1.K = n; x1.batch = cc;
      x1.A = GRbar; x1.sA = Nn; x1.ai = n; x1.ak = 1;
      x1.B = Gs + (long long)t0 * nn; x1.sB = nn; x1.bk = 1; x1.bj = n;
      x1.C = Xpart; x1.sC = Nn; x1.ci = n; x1.cj = 1;
      launch_gemm_f64(x1, s);
      GemmF64 x2 = x1;  // += sum_w GWtbar[j][P][w] G_j[w][p]
      x2.A = GWtbar; x2.bk = n; x2.bj = 1; x2.beta = 1.0;
      launch_gemm_f64(x2, s);
      GemmF64 m1;  // M1[j] = Ebar X    (N x n)
      m1.M = N; m1.Nc = n; m1.K = N; m1.batch = cc;
      m1.A = Sc; m1.sA = NN; m1.ai = N; m1.ak = 1;
      m1.B = X; m1.bk = n; m1.bj = 1;
      m1.C = M1; m1.sC = Nn; m1.ci = n; m1.cj = 1;
      launch_gemm_f64(m1, s);
      GemmF64 m2 = m1;  // M2[j] = Ebar^T X
      m2.ai = 1; m2.ak = N; m2.C = M2;
      launch_gemm_f64(m2, s);
      GemmF64 x3;  // Xpart += M1 Gm_j^T = -M1 G_{T-1-j}^T  : (P, r) <- sum_t M1[P][t] Gm[r][t]
      x3.M = N; x3.Nc = n; x3.K = n; x3.batch = cc;
      x3.A = M1; x3.sA = Nn; x3.ai = n; x3.ak = 1;
      x3.B = Gs + (long long)(T - 1 - t0) * nn; x3.sB = -nn; x3.bk = 1; x3.bj = n;
      x3.C = Xpart; x3.sC = Nn; x3.ci = n; x3.cj = 1;
      x3.alpha = -1.0; x3.beta = 1.0;
      launch_gemm_f64(x3, s);
      GemmF64 x4 = x3;  // Xpart += M2 Gm_j = -M2 G_{T-1-j} : (R, t) <- sum_r M2[R][r] Gm[r][t]
      x4.A = M2; x4.bk = n; x4.bj = 1;
      launch_gemm_f64(x4, s);
      k_sum_batches<<<grid1(Nn), 256, 0, s>>>(Xpart, Nn, cc, Xbar);
      launches += 8;
    }
  }
  // mixed tensors: Vbar = (U1bar + U2bar) Y^T; Z = V^T (U1bar + U2bar); Xbar from the pair products
  launch_add_f64(U1bar, U2bar, U1bar, Nn2, s);
  GemmF64 vb;
  vb.M = N; vb.Nc = N; vb.K = (int)nn;
  vb.A = U1bar; vb.ai = nn; vb.ak = 1;
  vb.B = Y; vb.bk = 1; vb.bj = nn;
  vb.C = Vbar; vb.ci = N; vb.cj = 1;
  launch_gemm_f64(vb, s);
  GemmF64 z;
  z.M = N; z.Nc = (int)nn; z.K = N;
  z.A = V; z.ai = 1; z.ak = N;
  z.B = U1bar; z.bk = nn; z.bj = 1;
  z.C = Z; z.ci = nn; z.cj = 1;
  launch_gemm_f64(z, s);
  k_pair_adjoint<<<grid1(Nn), 256, 0, s>>>(Z, X, N, n, Xbar);
  launches += 4;
  if (dX) SOX_CUDA_TRY(cudaMemcpyAsync(dX, Xbar, 8 * Nn, cudaMemcpyDeviceToDevice, s));
  if (dV) SOX_CUDA_TRY(cudaMemcpyAsync(dV, Vbar, 8 * NN, cudaMemcpyDeviceToDevice, s));
  h->launches += launches;
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

}  // namespace sox
