// Dynamically screened SOSEX for molecules in split precision (SOX_PREC_F16X2): the
// dynamic algorithm of Sec. II C (Eq. GG and the steps after it) with every contraction
// on the tensor cores as FP16-pair products with FP32 accumulation; the projections, the
// GG products and the final orbital-basis sum stay FP64.  W_d = W - v sits in slot U(1);
// SOX(v, v) comes from the static path.
//
// For every v (outer loop, as in the paper):
//   GG[j][(Q,u)]      = G_uQ(tau_j) G_Qv(-tau_j)                            FP64
//   GGw[m][c][(Q,u)]  = sum_j conj(T_fwd)[m][j]_c GG[j][(Q,u)]              FT GEMM, K = tau
//   Aw[m][c][P][u]    = sum_Q W_d[m][P][Q] GGw[m][c][Q][u]                  batched over (m, c)
//   A[i][v][(P,u)]    = sum_(m,c) T_inv[i][(m,c)] Aw[m][c][(P,u)]           IFT GEMM, K = (m, c)
// (the conjugated forward transform makes the real part of the inverse transform a plain
// real contraction over the interleaved (re, im) pairs of T_inv).  Then D[i] = sum_v
// (A[i][v] X^T) o (GWt_i U2_v^T) is the fused static kernel with X in the G_Rq slot, and
// Sigma_d = -X^T D^T X is added to Sigma.  GG, GGw and Aw are read in place as MN-major
// operands (gemm_mn.cu), each with one power-of-two scale per tensor.
#include <algorithm>

#include "dynamic.h"
#include "gemm_mn.h"
#include "tc_kernels.h"

namespace sox {
namespace {

int rup(long long x, int m) { return (int)((x + m - 1) / m * m); }
int grid1(long long total) { return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 65535 * 8)); }

// GG[j][Q][u] = GWt[j][Q][u] * (-GR[T-1-j][Q][v])
__global__ void k_gg_tc(const double *GWt, const double *GR, int T, int N, int n, int v, double *GG) {
  const long long Nn = (long long)N * n, total = Nn * T;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / Nn);
    const long long r = e % Nn;
    const int Q = (int)(r / n);
    GG[e] = -GWt[e] * GR[(long long)(T - 1 - j) * Nn + (long long)Q * n + v];
  }
}

// out = 1 / (a * b) for the scalars at a and b (device values)
__global__ void k_inv_prod(const float *a, const float *b, float *out) {
  *out = (float)(1.0 / ((double)*a * (double)*b));
}

// fill[i] = *src for i < count
__global__ void k_bcast(const float *src, float *fill, int count, float mul) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) fill[i] = *src * mul;
}

__global__ void k_fill1(float *p, int count, float v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) p[i] = v;
}

// scalars of the chain: split scales (written by the splits) and GEMM factors
struct DynScalars {
  float mx[8];     // atomicMax targets: Wd, Tf, Ti, GG, GGw, Aw, A
  float sc[8];     // scales of the same tensors
  float f[4];      // factors of the FT, W_d and IFT GEMMs
};
enum { kWd = 0, kTf, kTi, kGG, kGGw, kAw, kA };

struct DynGeom {
  int n, N, T, S, nO;
  int Kp, NR, Np, KpT, KpO;
  long long Nn4, Nn8;
  int np4, np8;
  int tc;          // tau points per chunk of the inverse transform and the fused kernel
};

DynGeom geom(sox_handle h, int n, int N, int T, int S, int nO) {
  DynGeom g{};
  g.n = n; g.N = N; g.T = T; g.S = S; g.nO = nO;
  g.Kp = rup(n, 64);
  g.NR = std::max(N, 128);
  g.Np = rup(N, 64);
  g.KpT = rup(T, 64);
  g.KpO = rup(2LL * nO, 64);
  g.Nn4 = ((long long)N * n + 3) & ~3LL;
  g.Nn8 = ((long long)N * n + 7) & ~7LL;
  g.np4 = rup(n, 4);
  g.np8 = rup(n, 8);
  // per tau point of a chunk: A in FP32 and as FP16 pairs (all v), the fused kernel's
  // operands and outputs
  const size_t per_t = (size_t)n * g.Nn4 * 4 + (size_t)n * g.NR * g.Kp * 4 + 4 * (size_t)g.NR * g.Kp +
                       (size_t)N * N * 4 + (size_t)N * n * 4 + 8 * (size_t)N + 4096;
  const size_t budget = chunk_budget(h, size_t(16) << 30);
  long long c = (long long)(budget / std::max<size_t>(per_t, 1));
  g.tc = (int)std::max<long long>(1, std::min<long long>(c, T));
  return g;
}

size_t fixed_bytes(const DynGeom &g) {
  const int n = g.n, N = g.N, T = g.T, nO = g.nO;
  size_t b = aligned_bytes((size_t)N * g.Kp * g.Kp, 4) + 2 * aligned_bytes((size_t)n * g.NR * g.Kp, 2) +
             aligned_bytes(N, 4);                                                     // U mixed, U2 split
  b += 2 * aligned_bytes((size_t)nO * N * g.Np, 2);                                   // W_d split
  b += 2 * aligned_bytes((size_t)2 * nO * g.KpT, 2) + 2 * aligned_bytes((size_t)T * g.KpO, 2);   // transforms
  b += 3 * aligned_bytes((size_t)T * N * n, 8);                                       // GR, GWt, GG
  b += 2 * aligned_bytes((size_t)T * g.NR * g.Kp, 2) + aligned_bytes((size_t)T * N, 4);   // GWt split
  b += 2 * aligned_bytes((size_t)T * g.NR * g.Kp, 2) + aligned_bytes((size_t)T * N, 4);   // X split per tau
  b += 2 * aligned_bytes((size_t)T * g.Nn8, 2);                                       // GG split
  b += aligned_bytes((size_t)2 * nO * g.Nn4, 4) + 2 * aligned_bytes((size_t)2 * nO * N * g.np8, 2);   // GGw
  b += aligned_bytes((size_t)2 * nO * N * g.np4, 4) + 2 * aligned_bytes((size_t)2 * nO * g.Nn8, 2);  // Aw
  b += aligned_bytes(sizeof(DynScalars), 4) + 4 * aligned_bytes((size_t)std::max(T, N), 4) + (1 << 16);
  return b;
}

size_t chunk_bytes(const DynGeom &g) {
  const int n = g.n, N = g.N, tc = g.tc;
  size_t b = aligned_bytes((size_t)tc * n * g.Nn4, 4);                                // A (FP32)
  b += 2 * aligned_bytes((size_t)tc * n * g.NR * g.Kp, 2);                            // A pairs
  b += 2 * aligned_bytes((size_t)tc * N, 4);                                          // row / col factors
  b += aligned_bytes((size_t)tc * N * N, 4) + aligned_bytes((size_t)tc * N * n, 4);   // Dt, T
  b += aligned_bytes((size_t)tc * n * n, 8);                                          // Sigma_d
  return b;
}

}  // namespace

size_t dynamic_tc_bytes(sox_handle h, int n, int N, int T, int S, int n_omega) {
  const DynGeom g = geom(h, n, N, T, S, n_omega);
  return fixed_bytes(g) + chunk_bytes(g) + (1 << 20);
}

Status dynamic_sigma_add_tc(sox_handle h, int n, int N, int T, int S, int n_omega, const double *G, const double *X,
                            const double *V, const double *Wd, const double *Tf, const double *Ti, double *Sigma,
                            Arena &ar, cudaStream_t s) {
  const DynGeom g = geom(h, n, N, T, S, n_omega);
  const int nO = n_omega, Kp = g.Kp, NR = g.NR;
  const long long nn = (long long)n * n, Nn = (long long)N * n;
  std::string err;
  // ---- buffers
  float *Um = ar.take<float>((size_t)N * Kp * Kp);
  __half *U2h = ar.take<__half>((size_t)n * NR * Kp), *U2l = ar.take<__half>((size_t)n * NR * Kp);
  float *inv_u2 = ar.take<float>(N);
  __half *Wh = ar.take<__half>((size_t)nO * N * g.Np), *Wl = ar.take<__half>((size_t)nO * N * g.Np);
  __half *Tfh = ar.take<__half>((size_t)2 * nO * g.KpT), *Tfl = ar.take<__half>((size_t)2 * nO * g.KpT);
  __half *Tih = ar.take<__half>((size_t)T * g.KpO), *Til = ar.take<__half>((size_t)T * g.KpO);
  double *GR = ar.take<double>((size_t)T * Nn), *GWt = ar.take<double>((size_t)T * Nn);
  double *GG = ar.take<double>((size_t)T * Nn);
  __half *GWh = ar.take<__half>((size_t)T * NR * Kp), *GWl = ar.take<__half>((size_t)T * NR * Kp);
  float *inv_gw = ar.take<float>((size_t)T * N);
  __half *Xh = ar.take<__half>((size_t)T * NR * Kp), *Xl = ar.take<__half>((size_t)T * NR * Kp);
  float *inv_x = ar.take<float>((size_t)T * N);
  __half *GGh = ar.take<__half>((size_t)T * g.Nn8), *GGl = ar.take<__half>((size_t)T * g.Nn8);
  float *GGw = ar.take<float>((size_t)2 * nO * g.Nn4);
  __half *GGwh = ar.take<__half>((size_t)2 * nO * N * g.np8), *GGwl = ar.take<__half>((size_t)2 * nO * N * g.np8);
  float *Aw = ar.take<float>((size_t)2 * nO * N * g.np4);
  __half *Awh = ar.take<__half>((size_t)2 * nO * g.Nn8), *Awl = ar.take<__half>((size_t)2 * nO * g.Nn8);
  DynScalars *sc = ar.take<DynScalars>(1);
  const int mT = std::max(T, N);
  float *ones = ar.take<float>(mT), *sAv = ar.take<float>(mT), *tmp1 = ar.take<float>(mT), *tmp2 = ar.take<float>(mT);
  const int tcn = g.tc;
  float *Af = ar.take<float>((size_t)tcn * n * g.Nn4);
  __half *Ah = ar.take<__half>((size_t)tcn * n * NR * Kp), *Al = ar.take<__half>((size_t)tcn * n * NR * Kp);
  float *rowf = ar.take<float>((size_t)tcn * N), *colf = ar.take<float>((size_t)tcn * N);
  float *Dt = ar.take<float>((size_t)tcn * N * N), *Tm = ar.take<float>((size_t)tcn * N * n);
  double *Sd = ar.take<double>((size_t)tcn * nn);
  if (!Sd) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  (void)tmp1;
  (void)tmp2;
  ProfScope ps(h, "sosex_dynamic_tc", s, 0);
  long long launches = 0;
  const long long limit = h->spin_limit;
  const int sms = h->sm_count;
  int v_lo = 0, v_hi = n;   // the handle's v range (sox_set_v_range)
  v_range(h, n, &v_lo, &v_hi);

  // ---- set-up: U2 = mixed tensor of V (per-P scale), W_d and the transforms (per tensor)
  SOX_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(DynScalars), s));
  SOX_CUDA_TRY(cudaMemsetAsync(U2h, 0, 2 * (size_t)n * NR * Kp, s));
  SOX_CUDA_TRY(cudaMemsetAsync(U2l, 0, 2 * (size_t)n * NR * Kp, s));
  launch_mixed_f32(V, X, N, n, Kp, Um, s);
  launch_split_mixed(Um, N, NR, n, Kp, nullptr, nullptr, U2h, U2l, inv_u2, s);
  launch_absmax(Wd, false, N, nO * N, 0, 1, 1, N, &sc->mx[kWd], s);
  launch_split_tensor(Wd, false, N, nO * N, 0, 1, 1, N, g.Np, 0, 1.f, &sc->mx[kWd], nullptr, Wh, Wl, &sc->sc[kWd], s);
  // forward transform conjugated: rows (m, 0) = Re T_fwd[m], rows (m, 1) = -Im T_fwd[m]
  launch_absmax(Tf, false, 2LL * T, nO, 0, 1, 1, 2 * T, &sc->mx[kTf], s);
  launch_split_tensor(Tf, false, 0, 1, 2LL * T, nO, 2, T, g.KpT, 2LL * g.KpT, 1.f, &sc->mx[kTf], nullptr, Tfh, Tfl,
                      &sc->sc[kTf], s);
  launch_split_tensor(Tf + 1, false, 0, 1, 2LL * T, nO, 2, T, g.KpT, 2LL * g.KpT, -1.f, &sc->mx[kTf], nullptr,
                      Tfh + g.KpT, Tfl + g.KpT, nullptr, s);
  // inverse transform: rows i, K = (m, c) the interleaved (re, im) pairs
  launch_absmax(Ti, false, 2LL * nO, T, 0, 1, 1, 2 * nO, &sc->mx[kTi], s);
  launch_split_tensor(Ti, false, 2LL * nO, T, 0, 1, 1, 2 * nO, g.KpO, 0, 1.f, &sc->mx[kTi], nullptr, Tih, Til,
                      &sc->sc[kTi], s);
  // X in the G_Rq slot, one copy per tau point (the fused kernel reads it at batch b)
  launch_split_rows_f64(X, n, 0, N, NR, n, Kp, Xh, Xl, inv_x, T, s);
  k_fill1<<<(mT + 255) / 256, 256, 0, s>>>(ones, mT, 1.f);
  launches += 13;

  // ---- tensor maps (fixed addresses)
  CUtensorMap mft[5], mwd[5], mbcd[8];
  if (!make_tmap_f16_3d_rs(&mft[0], Tfh, T, g.KpT, 2 * nO, 1, (uint64_t)2 * nO * g.KpT, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mft[1], Tfl, T, g.KpT, 2 * nO, 1, (uint64_t)2 * nO * g.KpT, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mft[2], GGh, Nn, g.Nn8, T, 1, (uint64_t)T * g.Nn8, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&mft[3], GGl, Nn, g.Nn8, T, 1, (uint64_t)T * g.Nn8, 64, 64, &err) ||
      !make_tmap_f32_store3d(&mft[4], GGw, Nn, 2 * nO, 1, g.Nn4, (uint64_t)2 * nO * g.Nn4, &err) ||
      !make_tmap_f16_3d_rs(&mwd[0], Wh, N, g.Np, N, nO, (uint64_t)N * g.Np, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mwd[1], Wl, N, g.Np, N, nO, (uint64_t)N * g.Np, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mwd[2], GGwh, n, g.np8, N, 2 * nO, (uint64_t)N * g.np8, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&mwd[3], GGwl, n, g.np8, N, 2 * nO, (uint64_t)N * g.np8, 64, 64, &err) ||
      !make_tmap_f32_store3d(&mwd[4], Aw, n, N, 2 * nO, g.np4, (uint64_t)N * g.np4, &err) ||
      !make_tmap_f16_3d(&mbcd[0], Ah, Kp, NR, (uint64_t)tcn * n, 64, 128, &err) ||
      !make_tmap_f16_3d(&mbcd[1], Al, Kp, NR, (uint64_t)tcn * n, 64, 128, &err) ||
      !make_tmap_f16_3d(&mbcd[2], Xh, Kp, NR, tcn, 64, 128, &err) ||
      !make_tmap_f16_3d(&mbcd[3], Xl, Kp, NR, tcn, 64, 128, &err) ||
      !make_tmap_f16_3d(&mbcd[4], GWh, Kp, NR, T, 64, 128, &err) ||
      !make_tmap_f16_3d(&mbcd[5], GWl, Kp, NR, T, 64, 128, &err) ||
      !make_tmap_f16_3d(&mbcd[6], U2h, Kp, NR, n, 64, 128, &err) ||
      !make_tmap_f16_3d(&mbcd[7], U2l, Kp, NR, n, 64, 128, &err))
    return {SOX_ERR_CUDA, "dynamic maps: " + err};

  for (int sp = 0; sp < S; ++sp) {
    const double *Gs = G + (long long)sp * T * nn;
    {  // GR[j][R][q] = sum_u X[R][u] G_j[u][q], GWt[j][P][w] = sum_p X[P][p] G_j[w][p]  (FP64)
      GemmF64 a;
      a.M = N; a.Nc = n; a.K = n; a.batch = T;
      a.A = X; a.ai = n; a.ak = 1;
      a.B = Gs; a.sB = nn; a.bk = n; a.bj = 1;
      a.C = GR; a.sC = Nn; a.ci = n; a.cj = 1;
      launch_gemm_f64(a, s);
      GemmF64 b = a;
      b.bk = 1; b.bj = n; b.C = GWt;
      launch_gemm_f64(b, s);
    }
    launch_split_rows_f64(GWt, n, Nn, N, NR, n, Kp, GWh, GWl, inv_gw, T, s);
    launches += 3;
    for (int i0 = 0; i0 < T; i0 += tcn) {
      const int ic = std::min(tcn, T - i0);
      CUtensorMap mift[5];
      if (!make_tmap_f16_3d_rs(&mift[0], Tih + (size_t)i0 * g.KpO, 2 * nO, g.KpO, ic, 1, (uint64_t)ic * g.KpO, 64, 128,
                               &err) ||
          !make_tmap_f16_3d_rs(&mift[1], Til + (size_t)i0 * g.KpO, 2 * nO, g.KpO, ic, 1, (uint64_t)ic * g.KpO, 64, 128,
                               &err) ||
          !make_tmap_f16_3d_rs(&mift[2], Awh, Nn, g.Nn8, 2 * nO, 1, (uint64_t)2 * nO * g.Nn8, 64, 64, &err) ||
          !make_tmap_f16_3d_rs(&mift[3], Awl, Nn, g.Nn8, 2 * nO, 1, (uint64_t)2 * nO * g.Nn8, 64, 64, &err))
        return {SOX_ERR_CUDA, "dynamic maps: " + err};
      for (int v = v_lo; v < v_hi; ++v) {
        SOX_CUDA_TRY(cudaMemsetAsync(&sc->mx[kGG], 0, 3 * sizeof(float), s));
        k_gg_tc<<<grid1((long long)T * Nn), 256, 0, s>>>(GWt, GR, T, N, n, v, GG);
        launch_absmax(GG, false, Nn, T, 0, 1, 1, (int)Nn, &sc->mx[kGG], s);
        launch_split_tensor(GG, false, Nn, T, 0, 1, 1, (int)Nn, g.Nn8, 0, 1.f, &sc->mx[kGG], nullptr, GGh, GGl,
                            &sc->sc[kGG], s);
        k_inv_prod<<<1, 1, 0, s>>>(&sc->sc[kTf], &sc->sc[kGG], &sc->f[0]);
        {  // GGw[(m,c)][(Q,u)] = sum_j conj(T_fwd)_c[m][j] GG[j][(Q,u)]
          GemmMnArgs a;
          a.M = 2 * nO; a.Ncols = (int)Nn; a.batch = 1; a.kc_inner = (T + 63) / 64; a.nk_outer = 1;
          a.a.mn_major = 0; a.b.mn_major = 1;
          a.alpha = &sc->f[0];
          a.spin_limit = limit; a.status = h->d_status;
          SOX_CUDA_TRY(launch_gemm_mn(mft, a, plan_gemm_mn(a, sms, 1), s));
        }
        launch_absmax(GGw, true, g.Nn4, 2 * nO, 0, 1, 1, (int)Nn, &sc->mx[kGGw], s);
        launch_split_tensor(GGw, true, n, N, g.Nn4, 2 * nO, 1, n, g.np8, (long long)N * g.np8, 1.f, &sc->mx[kGGw],
                            nullptr, GGwh, GGwl, &sc->sc[kGGw], s);
        k_inv_prod<<<1, 1, 0, s>>>(&sc->sc[kWd], &sc->sc[kGGw], &sc->f[1]);
        {  // Aw[(m,c)][P][u] = sum_Q W_d[m][P][Q] GGw[(m,c)][Q][u]
          GemmMnArgs a;
          a.M = N; a.Ncols = n; a.batch = 2 * nO; a.kc_inner = (N + 63) / 64; a.nk_outer = 1;
          a.a.mn_major = 0; a.a.zb = 1; a.a.zdiv = 2;
          a.b.mn_major = 1; a.b.zb = 1;
          a.alpha = &sc->f[1];
          a.spin_limit = limit; a.status = h->d_status;
          SOX_CUDA_TRY(launch_gemm_mn(mwd, a, plan_gemm_mn(a, sms, 1), s));
        }
        launch_absmax(Aw, true, g.np4, 2 * nO * N, 0, 1, 1, n, &sc->mx[kAw], s);
        launch_split_tensor(Aw, true, g.np4, N, (long long)N * g.np4, 2 * nO, 1, n, n, g.Nn8, 1.f, &sc->mx[kAw],
                            nullptr, Awh, Awl, &sc->sc[kAw], s);
        k_inv_prod<<<1, 1, 0, s>>>(&sc->sc[kTi], &sc->sc[kAw], &sc->f[2]);
        {  // A[i][v][(P,u)] = sum_(m,c) T_inv[i][(m,c)] Aw[(m,c)][(P,u)]  (i in this chunk)
          CUtensorMap mo;
          if (!make_tmap_f32_store3d(&mo, Af + (size_t)v * g.Nn4, Nn, ic, 1, (uint64_t)n * g.Nn4,
                                     (uint64_t)ic * n * g.Nn4, &err))
            return {SOX_ERR_CUDA, "dynamic maps: " + err};
          mift[4] = mo;
          GemmMnArgs a;
          a.M = ic; a.Ncols = (int)Nn; a.batch = 1; a.kc_inner = (2 * nO + 63) / 64; a.nk_outer = 1;
          a.a.mn_major = 0; a.b.mn_major = 1;
          a.alpha = &sc->f[2];
          a.spin_limit = limit; a.status = h->d_status;
          SOX_CUDA_TRY(launch_gemm_mn(mift, a, plan_gemm_mn(a, sms, 1), s));
        }
        launches += 14;
      }
      // A of the chunk as FP16 pairs [i][v][P][q] with one scale; then the fused B / C / D kernel
      SOX_CUDA_TRY(cudaMemsetAsync(&sc->mx[kA], 0, sizeof(float), s));
      SOX_CUDA_TRY(cudaMemsetAsync(Ah, 0, 2 * (size_t)ic * n * NR * Kp, s));
      SOX_CUDA_TRY(cudaMemsetAsync(Al, 0, 2 * (size_t)ic * n * NR * Kp, s));
      launch_absmax(Af, true, g.Nn4, ic * n, 0, 1, 1, (int)Nn, &sc->mx[kA], s);
      launch_split_tensor(Af, true, n, N, g.Nn4, ic * n, 1, n, Kp, (long long)NR * Kp, 1.f, &sc->mx[kA], nullptr, Ah,
                          Al, &sc->sc[kA], s);
      k_bcast<<<(ic + 255) / 256, 256, 0, s>>>(&sc->sc[kA], sAv, ic, 1.f);
      // D = acc * row[P] * col[R]: row = inv_gw[b][P] / s_A, col = inv_x[R] inv_u2[R]
      launch_bcd_scales(ones, sAv, ones, nullptr, NR, inv_gw + (size_t)i0 * N, inv_x, inv_u2, N, ic, rowf, colf, s);
      {
        CUtensorMap m[8] = {mbcd[0], mbcd[1], mbcd[2], mbcd[3], mbcd[4], mbcd[5], mbcd[6], mbcd[7]};
        if (!make_tmap_f16_3d(&m[4], GWh + (size_t)i0 * NR * Kp, Kp, NR, ic, 64, 128, &err) ||
            !make_tmap_f16_3d(&m[5], GWl + (size_t)i0 * NR * Kp, Kp, NR, ic, 64, 128, &err))
          return {SOX_ERR_CUDA, "dynamic maps: " + err};
        BcdArgs ba;
        ba.n = n; ba.N = N; ba.Kp = Kp; ba.batch = ic;
        ba.v0 = v_lo; ba.v1 = v_hi;
        ba.spin_limit = limit; ba.status = h->d_status;
        ba.row_scale = rowf; ba.col_scale = colf;
        ba.Dt = Dt; ba.ldD = N;
        const int tP = (N + 127) / 128;
        const int grid = (int)std::max<long long>(1, std::min<long long>((long long)ic * tP * tP, sms));
        ProfScope pb(h, "sox_bcd_dyn_tc", s);
        SOX_CUDA_TRY(launch_sox_bcd_tc(m, ba, grid, s, Kp <= 128 ? kBcdResident : kBcdStreamed));
      }
      // Sigma_d = -X^T D^T X (FP32 half transform, FP64 final sum), added to Sigma
      launch_backproject_T(Dt, N, X, N, n, ic, Tm, s);
      launch_backproject_sigma(X, Tm, N, n, ic, Sd, nn, s, nullptr);
      double *Sout = Sigma + ((long long)sp * T + i0) * nn;
      launch_add_f64(Sout, Sd, Sout, (long long)ic * nn, s);
      launches += 10;
    }
  }
  h->launches += launches;
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

}  // namespace sox
