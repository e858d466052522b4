// Adjoint of Phi_SOX with respect to X and V in split precision (SOX_PREC_F16X2):
// the reverse pass of the FP64 form (adjoint.cu) with every N x N x n contraction
// as an FP16-pair GEMM on the tensor cores (ctc.cu), FP32 results.
//
// Per spin and tau_j, c_j = -w_j dphi / 4, all v at once:
//   B_v = A_v GR^T,  C_v = GWt U2_v^T                     (recomputed)
//   Dbar = c_j E,  Bbar_v = Dbar o C_v,  Cbar_v = Dbar o B_v, Ebar = c_j sum_v B_v o C_v
//   Abar_v = Bbar_v GR,  GRbar = sum_v Bbar_v^T A_v,  GWtbar = sum_v Cbar_v U2_v,
//   U2bar_v += Cbar_v^T GWt,  U1bar += sum_v Abar_v (x) Gm_j[:, v]
// then Xbar from GRbar, GWtbar, Ebar (FP64), and at the end
//   Vbar = (U1bar + U2bar) Y^T,  Z = V^T (U1bar + U2bar),  Xbar += pair-product adjoint of Z.
#include <algorithm>

#include "adjoint.h"
#include "ctc.h"

namespace sox {
namespace {

long long rup4(long long x) { return (x + 3) & ~3LL; }
int grid1(long long total) { return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 65535 * 8)); }

// Dbar = c E and Ebar = c sum_v B_v o C_v (FP32, row length ld; the FP32 class of the split
// path), c = -w_j dphi / 4
__global__ void k_dbar(const float *B, const float *C, const float *E, const double *w, const double *dphi, int j,
                       int n, int N, long long ld, float *Dbar, float *Ebar) {
  const float c = (float)(-0.25 * w[j] * dphi[0]);
  const long long NN = (long long)N * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < NN; e += (long long)gridDim.x * blockDim.x) {
    const long long P = e / N, R = e % N, o = P * ld + R;
    float d = 0.f;
    for (int v = 0; v < n; ++v) d = fmaf(B[(long long)v * N * ld + o], C[(long long)v * N * ld + o], d);
    Dbar[o] = c * E[o];
    Ebar[o] = c * d;
  }
}

// out[r][q] (FP64, N x n) = sum_v in[v][r][q] (FP32, row length ld)
__global__ void k_sum_v(const float *in, int n, int N, long long ld, double *out) {
  const long long total = (long long)N * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n, q = e % n;
    double acc = 0.0;
    for (int v = 0; v < n; ++v) acc += (double)in[((long long)v * N + r) * ld + q];
    out[e] = acc;
  }
}

// Ubar[R][(a,b)] = U1bar[(R,a)][b] + U2bar[a][R][b]
__global__ void k_ubar(const float *U1bar, const float *U2bar, int n, int N, long long ld, long long ldU, float *Ubar) {
  const long long nn = (long long)n * n, total = (long long)N * nn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long R = e / nn, ab = e % nn, a = ab / n, b = ab % n;
    Ubar[R * ldU + ab] = U1bar[(R * n + a) * ld + b] + U2bar[(a * N + R) * ld + b];
  }
}

// Xbar[Q][q] += sum_s (Z[Q][(q,s)] + Z[Q][(s,q)]) X[Q][s]
__global__ void k_pair_adjoint_f32(const float *Z, long long ldZ, const double *X, int N, int n, double *Xbar) {
  const long long total = (long long)N * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long Q = e / n;
    const int q = (int)(e % n);
    const float *z = Z + Q * ldZ;
    const double *x = X + Q * n;
    double acc = 0.0;
    for (int s = 0; s < n; ++s) acc += ((double)z[q * n + s] + (double)z[s * n + q]) * x[s];
    Xbar[e] += acc;
  }
}

// out (FP64, rows x cols) = in (FP32, row length ld)
__global__ void k_to_f64(const float *in, long long ld, int rows, int cols, double *out) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (double)in[(e / cols) * ld + e % cols];
}

struct AdjGeom {
  int n, N, T, S;
  long long nn, np4, nnp, ldN, Nnp4;
};

AdjGeom adj_geom(int n, int N, int T, int S) {
  AdjGeom g{n, N, T, S};
  g.nn = (long long)n * n;
  g.np4 = rup4(n);
  g.nnp = rup4(g.nn);
  g.ldN = rup4(N);
  g.Nnp4 = rup4((long long)N * n);
  return g;
}

size_t setup_bytes(const AdjGeom &g) {
  const int n = g.n, N = g.N;
  return aligned_bytes((size_t)N * g.nn, 8) + rsplit_bytes(1, N, N) + rsplit_bytes(1, (int)g.nn, N) +
         aligned_bytes((size_t)N * g.nnp, 4) + rsplit_bytes(1, N * n, n) + rsplit_bytes(n, N, n) +
         rsplit_bytes(n, n, N) + aligned_bytes((size_t)N * n * g.np4, 4) + aligned_bytes((size_t)n * N * g.np4, 4) +
         aligned_bytes((size_t)N * n, 8) + rsplit_bytes(1, N, n) + rsplit_bytes(1, n, N);
}

size_t tau_bytes(const AdjGeom &g) {
  const int n = g.n, N = g.N;
  size_t b = 3 * aligned_bytes((size_t)N * n, 8) + aligned_bytes((size_t)N * g.ldN, 4);   // GR, GWt, M1, E
  b += 2 * rsplit_bytes(1, N, n) + 2 * rsplit_bytes(1, n, N) + 2 * rsplit_bytes(1, n, n);
  b += aligned_bytes((size_t)n * g.Nnp4, 4) + rsplit_bytes(n, N, n) + rsplit_bytes(n, n, N);
  b += 2 * aligned_bytes((size_t)n * N * g.ldN, 4) + 2 * aligned_bytes((size_t)N * g.ldN, 4);   // B, C, Dbar, Ebar
  b += rsplit_bytes(1, N, n) + 2 * rsplit_bytes(1, N, N) + 2 * aligned_bytes((size_t)N * g.np4, 4);   // E, Ebar X
  b += 4 * rsplit_bytes(n, N, N) + 3 * aligned_bytes((size_t)n * N * g.np4, 4) + rsplit_bytes(1, N * n, n);
  b += 4 * aligned_bytes((size_t)N * n, 8);   // GRbar, GWtbar, m1, m2
  return b;
}

size_t end_bytes(const AdjGeom &g) {
  const int N = g.N;
  return aligned_bytes((size_t)N * g.nnp, 4) + 2 * rsplit_bytes(1, N, (int)g.nn) + rsplit_bytes(1, N, N) +
         rsplit_bytes(1, (int)g.nn, N) + aligned_bytes((size_t)N * g.ldN, 4) + aligned_bytes((size_t)N * g.nnp, 4);
}

}  // namespace

size_t adjoint_tc_bytes(sox_handle, int n, int N, int T, int S) {
  const AdjGeom g = adj_geom(n, N, T, S);
  return setup_bytes(g) + std::max(tau_bytes(g), end_bytes(g)) + (1 << 20);
}

Status phi_adjoint_xv_tc(sox_handle h, int n, int N, int T, int S, const double *G, const double *X, const double *V,
                         const double *w, const double *dphi, double *dX, double *dV, Arena &ar, cudaStream_t s) {
  const AdjGeom g = adj_geom(n, N, T, S);
  const long long nn = g.nn, Nn = (long long)N * n, NN = (long long)N * N;
  // ---- set-up: mixed tensor in FP32 and its splits; accumulators
  double *Y = ar.take<double>((size_t)N * nn);
  CSplit Vs = rsplit_take(ar, 1, N, N), Ys = rsplit_take(ar, 1, (int)nn, N);
  float *Um = ar.take<float>((size_t)N * g.nnp);
  CSplit U1s = rsplit_take(ar, 1, N * n, n), U2v = rsplit_take(ar, n, N, n), U2vT = rsplit_take(ar, n, n, N);
  float *U1bar = ar.take<float>((size_t)N * n * g.np4), *U2bar = ar.take<float>((size_t)n * N * g.np4);
  double *Xbar = ar.take<double>((size_t)Nn);
  CSplit Xr = rsplit_take(ar, 1, N, n), XT = rsplit_take(ar, 1, n, N);   // X rows R (K = t); rows t (K = R)
  if (!Xbar || !U2vT.hi) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  ProfScope ps(h, "phi_adjoint_tc", s, 0);
  long long launches = 0;
  SOX_CUDA_TRY(cudaMemsetAsync(U1bar, 0, 4 * (size_t)N * n * g.np4, s));
  SOX_CUDA_TRY(cudaMemsetAsync(U2bar, 0, 4 * (size_t)n * N * g.np4, s));
  SOX_CUDA_TRY(cudaMemsetAsync(Xbar, 0, 8 * (size_t)Nn, s));
  launch_pair_products_f64(X, Y, N, n, s);
  rsplit(V, false, 0, N, 0, 0, 1, 1, N, N, Vs, s);
  rsplit(Y, false, 0, 1, 0, 0, nn, 1, (int)nn, N, Ys, s);                  // rows (a,b), K = Q
  SOX_TRY(cgemm_tc(h, Vs, Ys, 1, nullptr, nullptr, 1.f, Um, g.nnp, 0, s));   // Um[P][(a,b)]
  rsplit(Um, true, 0, g.nnp, n, n, 1, 1, N * n, n, U1s, s);                // rows (P,q), K = s
  rsplit(Um, true, n, g.nnp, 0, 0, 1, n, N, n, U2v, s);                    // [v] rows R, K = w
  rsplit(Um, true, n, 1, 0, 0, g.nnp, n, n, N, U2vT, s);                   // [v] rows w, K = R
  rsplit(X, false, 0, n, 0, 0, 1, 1, N, n, Xr, s);
  rsplit(X, false, 0, 1, 0, 0, n, 1, n, N, XT, s);
  launches += 8;

  // ---- per (spin, tau) buffers
  Arena at = ar;
  double *GR = at.take<double>(Nn), *GWt = at.take<double>(Nn), *M1 = at.take<double>(Nn);
  float *E = at.take<float>((size_t)N * g.ldN);
  CSplit M1s = rsplit_take(at, 1, N, n), Ebs = rsplit_take(at, 1, N, N), EbTs = rsplit_take(at, 1, N, N);
  float *m1f = at.take<float>((size_t)N * g.np4), *m2f = at.take<float>((size_t)N * g.np4);
  CSplit GRs = rsplit_take(at, 1, N, n), GWts = rsplit_take(at, 1, N, n);
  CSplit GRts = rsplit_take(at, 1, n, N), GWtts = rsplit_take(at, 1, n, N);
  CSplit Gma = rsplit_take(at, 1, n, n), Gmb = rsplit_take(at, 1, n, n);
  float *Aall = at.take<float>((size_t)n * g.Nnp4);
  CSplit As = rsplit_take(at, n, N, n), Ats = rsplit_take(at, n, n, N);
  float *Ball = at.take<float>((size_t)n * N * g.ldN), *Call = at.take<float>((size_t)n * N * g.ldN);
  float *Dbar = at.take<float>((size_t)N * g.ldN);
  float *Ebar = at.take<float>((size_t)N * g.ldN);
  CSplit Bbs = rsplit_take(at, n, N, N), Cbs = rsplit_take(at, n, N, N);
  CSplit BbTs = rsplit_take(at, n, N, N), CbTs = rsplit_take(at, n, N, N);
  float *Abar = at.take<float>((size_t)n * N * g.np4), *GRbv = at.take<float>((size_t)n * N * g.np4);
  float *GWbv = at.take<float>((size_t)n * N * g.np4);
  CSplit AbTs = rsplit_take(at, 1, N * n, n);
  double *GRbar = at.take<double>(Nn), *GWtbar = at.take<double>(Nn);
  double *m1 = at.take<double>(Nn), *m2 = at.take<double>(Nn);
  if (!m2 || !AbTs.hi) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  SOX_CUDA_TRY(cudaMemsetAsync(Ball, 0, 4 * (size_t)n * N * g.ldN, s));
  SOX_CUDA_TRY(cudaMemsetAsync(Call, 0, 4 * (size_t)n * N * g.ldN, s));
  SOX_CUDA_TRY(cudaMemsetAsync(Dbar, 0, 4 * (size_t)N * g.ldN, s));
  SOX_CUDA_TRY(cudaMemsetAsync(E, 0, 4 * (size_t)N * g.ldN, s));      // pad columns stay zero
  SOX_CUDA_TRY(cudaMemsetAsync(Ebar, 0, 4 * (size_t)N * g.ldN, s));

  for (int sp = 0; sp < S; ++sp) {
    for (int j = 0; j < T; ++j) {
      const double *Gj = G + ((long long)sp * T + j) * nn;
      const double *Gm = G + ((long long)sp * T + (T - 1 - j)) * nn;   // G(-tau_j) = -Gm
      {  // FP64 projections and E = X G(-tau_j) X^T
        GemmF64 a;
        a.M = N; a.Nc = n; a.K = n;
        a.A = X; a.ai = n; a.ak = 1;
        a.B = Gj; a.bk = n; a.bj = 1;
        a.C = GR; a.ci = n; a.cj = 1;
        launch_gemm_f64(a, s);
        GemmF64 b = a;
        b.bk = 1; b.bj = n; b.C = GWt;
        launch_gemm_f64(b, s);
        GemmF64 c = a;
        c.B = Gm; c.C = M1; c.alpha = -1.0;
        launch_gemm_f64(c, s);
      }
      rsplit(M1, false, 0, n, 0, 0, 1, 1, N, n, M1s, s);
      SOX_TRY(cgemm_tc(h, M1s, Xr, 1, nullptr, nullptr, 1.f, E, g.ldN, 0, s));   // E = X G(-tau_j) X^T
      rsplit(GR, false, 0, n, 0, 0, 1, 1, N, n, GRs, s);
      rsplit(GR, false, 0, 1, 0, 0, n, 1, n, N, GRts, s);
      rsplit(GWt, false, 0, n, 0, 0, 1, 1, N, n, GWts, s);
      rsplit(GWt, false, 0, 1, 0, 0, n, 1, n, N, GWtts, s);
      rsplit(Gm, false, 0, 1, 0, 0, n, 1, n, n, Gma, s);      // rows v, K = s: G(tau_{T-1-j})[s][v]
      rsplit(Gm, false, 0, n, 0, 0, 1, 1, n, n, Gmb, s);      // rows s, K = v
      // A_v[(P,q)] = -sum_s G(tau_{T-1-j})[s][v] U1[(P,q)][s]
      SOX_TRY(cgemm_tc(h, Gma, U1s, 1, nullptr, nullptr, -1.f, Aall, g.Nnp4, 0, s));
      rsplit(Aall, true, g.Nnp4, n, 0, 0, 1, n, N, n, As, s);    // [v] rows P, K = q
      rsplit(Aall, true, g.Nnp4, 1, 0, 0, n, n, n, N, Ats, s);   // [v] rows q, K = P
      SOX_TRY(cgemm_tc(h, As, GRs, n, nullptr, nullptr, 1.f, Ball, g.ldN, (long long)N * g.ldN, s));
      SOX_TRY(cgemm_tc(h, GWts, U2v, n, nullptr, nullptr, 1.f, Call, g.ldN, (long long)N * g.ldN, s));
      k_dbar<<<grid1(NN), 256, 0, s>>>(Ball, Call, E, w, dphi + sp, j, n, N, g.ldN, Dbar, Ebar);
      const long long sB = (long long)N * g.ldN;
      rsplit(Call, true, sB, g.ldN, 0, 0, 1, n, N, N, Bbs, s, Dbar);    // Bbar_v rows P, K = R
      rsplit(Ball, true, sB, g.ldN, 0, 0, 1, n, N, N, Cbs, s, Dbar);    // Cbar_v rows P, K = R
      rsplit(Call, true, sB, 1, 0, 0, g.ldN, n, N, N, BbTs, s, Dbar);   // Bbar_v^T rows R, K = P
      rsplit(Ball, true, sB, 1, 0, 0, g.ldN, n, N, N, CbTs, s, Dbar);   // Cbar_v^T rows R, K = P
      const long long sO = (long long)N * g.np4;
      SOX_TRY(cgemm_tc(h, Bbs, GRts, n, nullptr, nullptr, 1.f, Abar, g.np4, sO, s));   // Abar_v[P][q]
      SOX_TRY(cgemm_tc(h, BbTs, Ats, n, nullptr, nullptr, 1.f, GRbv, g.np4, sO, s));   // per-v GRbar[R][q]
      SOX_TRY(cgemm_tc(h, Cbs, U2vT, n, nullptr, nullptr, 1.f, GWbv, g.np4, sO, s));   // per-v GWtbar[P][w]
      SOX_TRY(cgemm_tc(h, CbTs, GWtts, n, nullptr, nullptr, 1.f, U2bar, g.np4, sO, s, true));   // U2bar_v[R][w]
      // U1bar[(P,q)][s] += -sum_v Abar_v[P][q] G(tau_{T-1-j})[s][v]
      rsplit(Abar, true, 0, g.np4, 1, n, sO, 1, N * n, n, AbTs, s);
      SOX_TRY(cgemm_tc(h, AbTs, Gmb, 1, nullptr, nullptr, -1.f, U1bar, g.np4, 0, s, true));
      k_sum_v<<<grid1(Nn), 256, 0, s>>>(GRbv, n, N, g.np4, GRbar);
      k_sum_v<<<grid1(Nn), 256, 0, s>>>(GWbv, n, N, g.np4, GWtbar);
      {  // Xbar += GRbar G_j^T + GWtbar G_j - (Ebar X) G_m^T - (Ebar^T X) G_m   (FP64)
        GemmF64 x1;
        x1.M = N; x1.Nc = n; x1.K = n;
        x1.A = GRbar; x1.ai = n; x1.ak = 1;
        x1.B = Gj; x1.bk = 1; x1.bj = n;
        x1.C = Xbar; x1.ci = n; x1.cj = 1; x1.beta = 1.0;
        launch_gemm_f64(x1, s);
        GemmF64 x2 = x1;
        x2.A = GWtbar; x2.bk = n; x2.bj = 1;
        launch_gemm_f64(x2, s);
        // m1 = Ebar X, m2 = Ebar^T X on the tensor cores
        rsplit(Ebar, true, 0, g.ldN, 0, 0, 1, 1, N, N, Ebs, s);
        rsplit(Ebar, true, 0, 1, 0, 0, g.ldN, 1, N, N, EbTs, s);
        SOX_TRY(cgemm_tc(h, Ebs, XT, 1, nullptr, nullptr, 1.f, m1f, g.np4, 0, s));
        SOX_TRY(cgemm_tc(h, EbTs, XT, 1, nullptr, nullptr, 1.f, m2f, g.np4, 0, s));
        k_to_f64<<<grid1(Nn), 256, 0, s>>>(m1f, g.np4, N, n, m1);
        k_to_f64<<<grid1(Nn), 256, 0, s>>>(m2f, g.np4, N, n, m2);
        GemmF64 x3;
        x3.M = N; x3.Nc = n; x3.K = n;
        x3.A = m1; x3.ai = n; x3.ak = 1;
        x3.B = Gm; x3.bk = 1; x3.bj = n;
        x3.C = Xbar; x3.ci = n; x3.cj = 1;
        x3.alpha = -1.0; x3.beta = 1.0;
        launch_gemm_f64(x3, s);
        GemmF64 x4 = x3;
        x4.A = m2; x4.bk = n; x4.bj = 1;
        launch_gemm_f64(x4, s);
      }
      launches += 4 + 6 + 2 + 1 + 4 + 1 + 2 + 6;
    }
  }

  // ---- end: Ubar = U1bar + U2bar; Vbar = Ubar Y^T; Z = V^T Ubar; Xbar += pair adjoint of Z
  Arena ae = ar;
  float *Ubar = ae.take<float>((size_t)N * g.nnp);
  CSplit Ubs = rsplit_take(ae, 1, N, (int)nn), Yr = rsplit_take(ae, 1, N, (int)nn);
  CSplit VTs = rsplit_take(ae, 1, N, N), UbTs = rsplit_take(ae, 1, (int)nn, N);
  float *Vbar = ae.take<float>((size_t)N * g.ldN), *Z = ae.take<float>((size_t)N * g.nnp);
  if (!Z || !UbTs.hi) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  k_ubar<<<grid1((long long)N * nn), 256, 0, s>>>(U1bar, U2bar, n, N, g.np4, g.nnp, Ubar);
  rsplit(Ubar, true, 0, g.nnp, 0, 0, 1, 1, N, (int)nn, Ubs, s);
  rsplit(Y, false, 0, nn, 0, 0, 1, 1, N, (int)nn, Yr, s);
  SOX_TRY(cgemm_tc(h, Ubs, Yr, 1, nullptr, nullptr, 1.f, Vbar, g.ldN, 0, s));
  rsplit(V, false, 0, 1, 0, 0, N, 1, N, N, VTs, s);                 // rows Q, K = P
  rsplit(Ubar, true, 0, 1, 0, 0, g.nnp, 1, (int)nn, N, UbTs, s);    // rows (a,b), K = P
  SOX_TRY(cgemm_tc(h, VTs, UbTs, 1, nullptr, nullptr, 1.f, Z, g.nnp, 0, s));
  k_pair_adjoint_f32<<<grid1(Nn), 256, 0, s>>>(Z, g.nnp, X, N, n, Xbar);
  if (dV) k_to_f64<<<grid1(NN), 256, 0, s>>>(Vbar, g.ldN, N, N, dV);
  if (dX) SOX_CUDA_TRY(cudaMemcpyAsync(dX, Xbar, 8 * (size_t)Nn, cudaMemcpyDeviceToDevice, s));
  launches += 9;
  h->launches += launches;
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

}  // namespace sox
