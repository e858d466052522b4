// Static SOX for periodic solids (Sec. II C, the algorithm with momenta), FP64
// complex on CUDA cores.
//
// For the external momentum k and transfers q1, q2 (labels k - q with q = k_i - k_j):
//   M^{q,k'}[P][a][b] = sum_Q U^q_PQ conj(X^{k'-q}_{aQ}) X^{k'}_{bQ}        (mixed tensors)
//   GR^k = X^k G^k,  GWt^k[P][w] = sum_p conj(X^k[P][p]) G^k[w][p]
//   A^{q1,ks}[v][P][q] = sum_s G^{ks}(-tau)[s][v] M^{q1,ks}[P][q][s]
//   B^{q1,ks}_v[P][R]  = sum_q A^{q1,ks}[v][P][q] GR^{ks-q1}[R][q]             (regime 1)
//   C^{q2,kw}_v[P][R]  = sum_w GWt^{kw}[P][w] M^{q2,kw}[R][v][w]               (regime 1)
//   D^k[P][R] = sum_{q1,q2} sum_v C^{q2,k+q1}_v[P][R] B^{q1,k+q1-q2}_v[P][R]    (regime 2)
//   Sigma^k[t][r] = -1/N_k^2 sum_R conj(X^k[R][t]) sum_P D^k[P][R] X^k[P][r]
// B and C for every (q, k') pair are produced for a chunk of v at a time.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctc.h"
#include "kpoint.h"

namespace sox {
namespace {

using z = double2;
__device__ __forceinline__ z zmul(z a, z b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ z zfma(z a, z b, z c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ z zconj(z a) { return make_double2(a.x, -a.y); }

constexpr int TM = 64, TK = 8, NT = 256;

// Grouped complex GEMM: C[b](i,j) = alpha sum_k opA(i,k) opB(k,j) + beta C[b](i,j),
// opX = conj(X) when conjX; batch b at base + (off ? off[b] : b * stride) elements.
struct ZGemm {
  int M, Nc, K, batch;
  const z *A; long long sA, ai, ak; const long long *offA; int conjA;
  const z *B; long long sB, bk, bj; const long long *offB; int conjB;
  z *C; long long sC, ci, cj; const long long *offC;
  double alpha, beta;
};

__global__ void __launch_bounds__(NT) k_zgemm(ZGemm g) {
  __shared__ z sa[TK][TM + 1];
  __shared__ z sb[TK][TM + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TM;
  const long long b = blockIdx.z;
  const z *A = g.A + (g.offA ? g.offA[b] : b * g.sA);
  const z *B = g.B + (g.offB ? g.offB[b] : b * g.sB);
  z *C = g.C + (g.offC ? g.offC[b] : b * g.sC);
  z acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < g.K; k0 += TK) {
#pragma unroll
    for (int it = 0; it < (TM * TK) / NT; ++it) {
      const int e = tid + it * NT;
      int r, k;
      if (g.ak == 1) { r = e / TK; k = e % TK; } else { r = e % TM; k = e / TM; }
      const int gr = i0 + r, gk = k0 + k;
      z v = make_double2(0.0, 0.0);
      if (gr < g.M && gk < g.K) v = A[gr * g.ai + gk * g.ak];
      sa[k][r] = g.conjA ? zconj(v) : v;
      int c, kb;
      if (g.bj == 1) { c = e % TM; kb = e / TM; } else { c = e / TK; kb = e % TK; }
      const int gc = j0 + c, gkb = k0 + kb;
      z w = make_double2(0.0, 0.0);
      if (gc < g.Nc && gkb < g.K) w = B[gkb * g.bk + gc * g.bj];
      sb[kb][c] = g.conjB ? zconj(w) : w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      z av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = sa[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = sb[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = zfma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = i0 + ty + 16 * i;
    if (gi >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = j0 + tx + 16 * j;
      if (gj >= g.Nc) continue;
      z *c = C + gi * g.ci + gj * g.cj;
      z v = make_double2(g.alpha * acc[i][j].x, g.alpha * acc[i][j].y);
      if (g.beta != 0.0) v = make_double2(v.x + g.beta * c->x, v.y + g.beta * c->y);
      *c = v;
    }
  }
}

void zgemm(const ZGemm &g, cudaStream_t s) {
  if (g.M <= 0 || g.Nc <= 0 || g.batch <= 0) return;
  dim3 grid((g.Nc + TM - 1) / TM, (g.M + TM - 1) / TM, g.batch);
  k_zgemm<<<grid, NT, 0, s>>>(g);
}

ZGemm zg() {
  ZGemm g{};
  g.batch = 1;
  g.alpha = 1.0;
  return g;
}

// Y[pair][Q][a][b] = conj(X[k'-q][Q][a]) X[k'][Q][b] for every (q, k') pair
__global__ void k_kpair_products(const z *X, const int *sub, int nk, int N, int n, z *Y) {
  const long long per = (long long)N * n * n;
  const long long total = per * nk * nk;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int pair = (int)(e / per);
    const long long r = e % per;
    const int Q = (int)(r / ((long long)n * n));
    const int a = (int)((r / n) % n), bb = (int)(r % n);
    const int q = pair / nk, kk = pair % nk;
    const int ka = sub[kk * nk + q];
    Y[e] = zmul(zconj(X[((long long)ka * N + Q) * n + a]), X[((long long)kk * N + Q) * n + bb]);
  }
}

// D[k][P][R] += sum_{q1,q2} sum_{v<nv} C[(q2, k+q1)][v][P][R] * B[(q1, k+q1-q2)][v][P][R]
__global__ void k_kpoint_D(const z *B, const z *C, const int *add, const int *sub, int nk, int N, int nv,
                           z *D) {
  const int R = blockIdx.x * 32 + threadIdx.x;
  const int P = blockIdx.y * 8 + threadIdx.y;
  const int k = blockIdx.z;
  if (P >= N || R >= N) return;
  const long long NN = (long long)N * N, pe = (long long)P * N + R;
  z acc = D[(long long)k * NN + pe];
  for (int q1 = 0; q1 < nk; ++q1) {
    const int kw = add[k * nk + q1];
    for (int q2 = 0; q2 < nk; ++q2) {
      const int ks = sub[kw * nk + q2];
      const z *c = C + ((long long)(q2 * nk + kw) * nv) * NN + pe;
      const z *b = B + ((long long)(q1 * nk + ks) * nv) * NN + pe;
      for (int v = 0; v < nv; ++v) acc = zfma(c[v * NN], b[v * NN], acc);
    }
  }
  D[(long long)k * NN + pe] = acc;
}

int grid1(long long total) { return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 65535 * 8)); }

// add[a][b] = index of k_a + k_b, sub[a][b] = index of k_a - k_b on the problem's mesh
void mesh_tables(const sox_problem *pr, std::vector<int> &add, std::vector<int> &sub) {
  const int n1 = pr->nk[0], n2 = pr->nk[1], n3 = pr->nk[2], nk = n1 * n2 * n3;
  add.assign((size_t)nk * nk, 0);
  sub.assign((size_t)nk * nk, 0);
  auto idx = [&](int x, int y, int zz) {
    x = ((x % n1) + n1) % n1;
    y = ((y % n2) + n2) % n2;
    zz = ((zz % n3) + n3) % n3;
    return (x * n2 + y) * n3 + zz;
  };
  for (int a = 0; a < nk; ++a)
    for (int b = 0; b < nk; ++b) {
      const int ax = a / (n2 * n3), ay = (a / n3) % n2, az = a % n3;
      const int bx = b / (n2 * n3), by = (b / n3) % n2, bz = b % n3;
      add[(size_t)a * nk + b] = idx(ax + bx, ay + by, az + bz);
      sub[(size_t)a * nk + b] = idx(ax - bx, ay - by, az - bz);
    }
}

// GG[ks][j][Q][u] = GWt[ku][j][Q][u] * (-GR[ks][T-1-j][Q][v]),  ku = ks - q1
__global__ void k_gg_k(const z *GWt, const z *GR, const int *sub, int nk, int q1, int T, int N, int n, int v, z *GG) {
  const long long Nn = (long long)N * n, per = Nn * T, total = per * nk;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int ks = (int)(e / per);
    const long long r = e % per;
    const int j = (int)(r / Nn);
    const long long qu = r % Nn;
    const int Q = (int)(qu / n);
    const int ku = sub[ks * nk + q1];
    const z a = GWt[((long long)ku * T + j) * Nn + qu];
    const z g = GR[((long long)ks * T + (T - 1 - j)) * Nn + (long long)Q * n + v];
    GG[e] = zmul(a, make_double2(-g.x, -g.y));
  }
}

// D[i][k][P][R] += sum_{q1,q2} C[(q2, k+q1)][il][P][R] * B[(q1, k+q1-q2)][il][P][R],  i = i0 + il
__global__ void k_kpoint_D_tau(const z *B, const z *C, const int *add, const int *sub, int nk, int N, int ct, int i0,
                               z *D) {
  const int R = blockIdx.x * 32 + threadIdx.x;
  const int P = blockIdx.y * 8 + threadIdx.y;
  const int k = blockIdx.z % nk, il = blockIdx.z / nk;
  if (P >= N || R >= N) return;
  const long long NN = (long long)N * N, pe = (long long)P * N + R;
  z *d = D + ((long long)(i0 + il) * nk + k) * NN + pe;
  z acc = *d;
  for (int q1 = 0; q1 < nk; ++q1) {
    const int kw = add[k * nk + q1];
    for (int q2 = 0; q2 < nk; ++q2) {
      const int ks = sub[kw * nk + q2];
      acc = zfma(C[((long long)(q2 * nk + kw) * ct + il) * NN + pe], B[((long long)(q1 * nk + ks) * ct + il) * NN + pe],
                 acc);
    }
  }
  *d = acc;
}

}  // namespace

KpointPlan kpoint_plan(sox_handle h, int n, int N, int T, int S, const int nkv[3]) {
  KpointPlan p{};
  p.nk = nkv[0] * nkv[1] * nkv[2];
  const size_t nk2 = (size_t)p.nk * p.nk;
  const size_t Nn2 = (size_t)N * n * n, NN = (size_t)N * N, Nn = (size_t)N * n;
  p.fixed_bytes = 16 * (2 * nk2 * Nn2 /*Y, M*/ + (size_t)p.nk * (2 * Nn + NN + Nn) /*GR, GWt, D, T*/) +
                  8 * 2 * nk2 /*tables*/ + 64 * 1024;
  const size_t per_v = 16 * nk2 * (2 * NN /*B, C*/ + Nn /*A*/);
  const size_t budget = chunk_budget(h, size_t(24) << 30);
  long long nv = budget > p.fixed_bytes ? (long long)((budget - p.fixed_bytes) / per_v) : 1;
  p.nv = (int)std::max<long long>(1, std::min<long long>(nv, n));
  p.bytes = p.fixed_bytes + per_v * p.nv + 16 * (size_t)3 * nk2 * p.nv * sizeof(long long) + 64 * 1024;
  (void)T;
  (void)S;
  return p;
}

Status kpoint_sigma_f64(sox_handle h, const sox_problem *pr, const double *Gd, const double *Xd, const double *U1d,
                        const double *U2d, double *Sd, Arena &ar, cudaStream_t s) {
  int v_lo = 0, v_hi = pr->n;   // the handle's v range (sox_set_v_range)
  v_range(h, pr->n, &v_lo, &v_hi);
  const int n = pr->n, N = pr->N, T = pr->n_tau, S = pr->n_spin;
  const KpointPlan pl = kpoint_plan(h, n, N, T, S, pr->nk);
  const int nk = pl.nk, nv = pl.nv;
  const long long nn = (long long)n * n, Nn2 = (long long)N * nn, NN = (long long)N * N, Nn = (long long)N * n;
  const long long nk2 = (long long)nk * nk;
  const z *G = reinterpret_cast<const z *>(Gd);
  const z *X = reinterpret_cast<const z *>(Xd);
  const z *U1 = reinterpret_cast<const z *>(U1d);
  const z *U2 = reinterpret_cast<const z *>(U2d);
  z *Sig = reinterpret_cast<z *>(Sd);
  const bool two = (U1d != U2d);

  // momentum tables (host -> device, through the workspace)
  std::vector<int> add(nk * nk), sub(nk * nk);
  {
    std::vector<int> m(3 * nk);
    for (int a = 0; a < nk; ++a) {
      m[3 * a + 0] = a / (pr->nk[1] * pr->nk[2]);
      m[3 * a + 1] = (a / pr->nk[2]) % pr->nk[1];
      m[3 * a + 2] = a % pr->nk[2];
    }
    auto idx = [&](int x, int y, int zz) {
      x = ((x % pr->nk[0]) + pr->nk[0]) % pr->nk[0];
      y = ((y % pr->nk[1]) + pr->nk[1]) % pr->nk[1];
      zz = ((zz % pr->nk[2]) + pr->nk[2]) % pr->nk[2];
      return (x * pr->nk[1] + y) * pr->nk[2] + zz;
    };
    for (int a = 0; a < nk; ++a)
      for (int b = 0; b < nk; ++b) {
        add[a * nk + b] = idx(m[3 * a] + m[3 * b], m[3 * a + 1] + m[3 * b + 1], m[3 * a + 2] + m[3 * b + 2]);
        sub[a * nk + b] = idx(m[3 * a] - m[3 * b], m[3 * a + 1] - m[3 * b + 1], m[3 * a + 2] - m[3 * b + 2]);
      }
  }
  int *d_add = ar.take<int>(nk2), *d_sub = ar.take<int>(nk2);
  z *Y = ar.take<z>(nk2 * Nn2), *M1 = ar.take<z>(nk2 * Nn2);
  z *M2 = two ? ar.take<z>(nk2 * Nn2) : M1;
  z *GR = ar.take<z>((size_t)nk * Nn), *GWt = ar.take<z>((size_t)nk * Nn);
  z *D = ar.take<z>((size_t)nk * NN), *Tm = ar.take<z>((size_t)nk * Nn);
  z *A = ar.take<z>((size_t)nk2 * nv * Nn);
  z *Bc = ar.take<z>((size_t)nk2 * nv * NN), *Cc = ar.take<z>((size_t)nk2 * nv * NN);
  long long *offA = ar.take<long long>(nk2 * nv), *offB = ar.take<long long>(nk2 * nv);
  long long *offC = ar.take<long long>(nk2 * nv), *offD = ar.take<long long>(nk2 * nv);
  if (!offD) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  SOX_CUDA_TRY(cudaMemcpyAsync(d_add, add.data(), 4 * nk2, cudaMemcpyHostToDevice, s));
  SOX_CUDA_TRY(cudaMemcpyAsync(d_sub, sub.data(), 4 * nk2, cudaMemcpyHostToDevice, s));
  ProfScope ps(h, "kpoint_f64", s, 0);
  long long launches = 0;

  // mixed tensors for every (q, k'): M[q][k'] = U^q Y[q][k']   (Y as [Q][(a,b)])
  auto mixed = [&](const z *U, z *Mout) {
    for (int q = 0; q < nk; ++q) {
      ZGemm g = zg();
      g.M = N; g.Nc = (int)nn; g.K = N; g.batch = nk;
      g.A = U + (long long)q * NN; g.ai = N; g.ak = 1;
      g.B = Y + (long long)q * nk * Nn2; g.sB = Nn2; g.bk = nn; g.bj = 1;
      g.C = Mout + (long long)q * nk * Nn2; g.sC = Nn2; g.ci = nn; g.cj = 1;
      zgemm(g, s);
      ++launches;
    }
  };
  k_kpair_products<<<grid1(nk2 * Nn2), 256, 0, s>>>(X, d_sub, nk, N, n, Y);
  ++launches;
  mixed(U1, M1);
  if (two) mixed(U2, M2);

  // offset tables for the grouped GEMMs of one v-chunk (host-built, uploaded once per chunk shape)
  std::vector<long long> hA(nk2 * nv), hB(nk2 * nv), hC(nk2 * nv), hD(nk2 * nv);
  const double inv_nk2 = 1.0 / ((double)nk * nk);
  for (int sp = 0; sp < S; ++sp) {
    for (int j = 0; j < T; ++j) {
      const z *Gj = G + ((long long)sp * nk * T) * nn;   // G[sp][k][t] at + (k*T + t)*nn
      // projections for every k at tau_j
      {
        ZGemm g = zg();  // GR[k] = X[k] G[k](tau_j)
        g.M = N; g.Nc = n; g.K = n; g.batch = nk;
        g.A = X; g.sA = Nn; g.ai = n; g.ak = 1;
        g.B = Gj + (long long)j * nn; g.sB = (long long)T * nn; g.bk = n; g.bj = 1;
        g.C = GR; g.sC = Nn; g.ci = n; g.cj = 1;
        zgemm(g, s);
        ZGemm w = g;     // GWt[k][P][w] = sum_p conj(X[k][P][p]) G[k][w][p]
        w.conjA = 1; w.bk = 1; w.bj = n; w.C = GWt;
        zgemm(w, s);
        launches += 2;
      }
      SOX_CUDA_TRY(cudaMemsetAsync(D, 0, 16 * (size_t)nk * NN, s));
      for (int v0 = v_lo; v0 < v_hi; v0 += nv) {   // the handle's v range (sox_set_v_range)
        const int cv = std::min(nv, v_hi - v0);
        // A[pair][vl][P][q] = -sum_s G^{k'}(tau_{T-1-j})[s][v0+vl] M1[pair][P][q][s]
        for (int q = 0; q < nk; ++q) {
          ZGemm g = zg();
          g.M = cv; g.Nc = N * n; g.K = n; g.batch = nk;
          g.A = Gj + (long long)(T - 1 - j) * nn + v0; g.sA = (long long)T * nn; g.ai = 1; g.ak = n;
          g.B = M1 + (long long)q * nk * Nn2; g.sB = Nn2; g.bk = 1; g.bj = n;
          g.C = A + (long long)q * nk * cv * Nn; g.sC = (long long)cv * Nn; g.ci = Nn; g.cj = 1;
          g.alpha = -1.0;
          zgemm(g, s);
          ++launches;
        }
        // B[pair][vl][P][R] = sum_q A[pair][vl][P][q] GR[k'-q1][R][q]     (grouped over pair, vl)
        // C[pair][vl][P][R] = sum_w GWt[k'][P][w] M2[pair][R][v][w]      (grouped over pair, vl)
        for (int q = 0; q < nk; ++q)
          for (int kk = 0; kk < nk; ++kk)
            for (int vl = 0; vl < cv; ++vl) {
              const long long b = ((long long)q * nk + kk) * cv + vl;
              hA[b] = (((long long)q * nk + kk) * cv + vl) * Nn;       // A slice
              hB[b] = (long long)sub[kk * nk + q] * Nn;                 // GR[k'-q]
              hC[b] = (long long)kk * Nn;                               // GWt[k']
              hD[b] = ((long long)q * nk + kk) * Nn2 + (long long)(v0 + vl) * n;  // M2[pair][.][v][.]
            }
        const long long nb = nk2 * cv;
        SOX_CUDA_TRY(cudaMemcpyAsync(offA, hA.data(), 8 * nb, cudaMemcpyHostToDevice, s));
        SOX_CUDA_TRY(cudaMemcpyAsync(offB, hB.data(), 8 * nb, cudaMemcpyHostToDevice, s));
        SOX_CUDA_TRY(cudaMemcpyAsync(offC, hC.data(), 8 * nb, cudaMemcpyHostToDevice, s));
        SOX_CUDA_TRY(cudaMemcpyAsync(offD, hD.data(), 8 * nb, cudaMemcpyHostToDevice, s));
        ZGemm gb = zg();
        gb.M = N; gb.Nc = N; gb.K = n; gb.batch = (int)nb;
        gb.A = A; gb.offA = offA; gb.ai = n; gb.ak = 1;
        gb.B = GR; gb.offB = offB; gb.bk = 1; gb.bj = n;
        gb.C = Bc; gb.sC = NN; gb.ci = N; gb.cj = 1;
        zgemm(gb, s);
        ZGemm gc = zg();
        gc.M = N; gc.Nc = N; gc.K = n; gc.batch = (int)nb;
        gc.A = GWt; gc.offA = offC; gc.ai = n; gc.ak = 1;
        gc.B = M2; gc.offB = offD; gc.bk = 1; gc.bj = nn;
        gc.C = Cc; gc.sC = NN; gc.ci = N; gc.cj = 1;
        zgemm(gc, s);
        {
          dim3 grid((N + 31) / 32, (N + 7) / 8, nk);
          k_kpoint_D<<<grid, dim3(32, 8), 0, s>>>(Bc, Cc, d_add, d_sub, nk, N, cv, D);
        }
        launches += 3;
        // (the host tables may be rewritten now: a copy from pageable memory returns only
        // once the host buffer has been staged, and stream order protects the device tables)
      }
      // Sigma^k = -1/N_k^2 X^H D^T X :  T[k][R][r] = sum_P D[k][P][R] X[k][P][r]
      ZGemm t = zg();
      t.M = N; t.Nc = n; t.K = N; t.batch = nk;
      t.A = D; t.sA = NN; t.ai = 1; t.ak = N;
      t.B = X; t.sB = Nn; t.bk = n; t.bj = 1;
      t.C = Tm; t.sC = Nn; t.ci = n; t.cj = 1;
      zgemm(t, s);
      ZGemm o = zg();  // Sigma[sp][k][j][t][r] = -1/N_k^2 sum_R conj(X[k][R][t]) T[k][R][r]
      o.M = n; o.Nc = n; o.K = N; o.batch = nk;
      o.A = X; o.sA = Nn; o.ai = 1; o.ak = n; o.conjA = 1;
      o.B = Tm; o.sB = Nn; o.bk = n; o.bj = 1;
      o.C = Sig + ((long long)sp * nk * T + j) * nn; o.sC = (long long)T * nn; o.ci = n; o.cj = 1;
      o.alpha = -inv_nk2;
      zgemm(o, s);
      launches += 2;
    }
  }
  h->launches += launches;
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

// ---------------------------------------------------------------------------
// Dynamically screened SOSEX for solids: adds Sigma_d to Sigma (which holds SOX(v, v)).
// W_d^{q1}(i Omega) in slot U(1), bare v in U(2); for every v and (q1, k_s):
//   GG_Quv(tau_j) = G^{k_u}_uQ(tau_j) G^{k_s}_Qv(-tau_j),  k_u = k_s - q1
//   A_Puv(tau_i)  = sum_m T_inv[i][m] sum_Q W_d^{q1}_PQ(i Omega_m) sum_j T_fwd[m][j] GG_Quv(tau_j)
//   B^{q1,ks}_v(tau_i)[P][R] = sum_u A_Puv(tau_i) X^{k_u}[R][u]
// then C and the n_k^3 D step per tau_i, and Sigma^k_d = -1/N_k^2 X_k^H D^T X_k.
// ---------------------------------------------------------------------------
size_t kpoint_dynamic_bytes(sox_handle h, int n, int N, int T, int n_omega, const int nkv[3], int *ct_out) {
  const size_t nk = (size_t)nkv[0] * nkv[1] * nkv[2], nk2 = nk * nk;
  const size_t Nn2 = (size_t)N * n * n, NN = (size_t)N * N, Nn = (size_t)N * n;
  const size_t fixed = 16 * (2 * nk2 * Nn2 /*Y, M*/ + 3 * nk * T * Nn /*GWt, GR, GG*/ + 2 * nk * n_omega * Nn /*GGw, Aw*/ +
                             nk2 * T * Nn /*A*/ + (size_t)T * nk * NN /*D*/ + 2 * nk * Nn /*T1*/) +
                       8 * 3 * nk2 * n_omega /*offsets of the W product*/ + 64 * 1024;
  const size_t per_t = 16 * 2 * nk2 * NN + 8 * 4 * nk2;
  const size_t budget = chunk_budget(h, size_t(32) << 30);
  long long ct = budget > fixed ? (long long)((budget - fixed) / per_t) : 1;
  ct = std::min<long long>(ct, 65535 / (long long)nk2);  // grouped-GEMM batch is a grid dimension
  ct = std::max<long long>(1, std::min<long long>(ct, T));
  if (ct_out) *ct_out = (int)ct;
  return fixed + per_t * ct + 64 * 1024;
}

Status kpoint_dynamic_add_f64(sox_handle h, const sox_problem *pr, int n_omega, const double *Gd, const double *Xd,
                              const double *Vd, const double *Wdd, const double *Tfd, const double *Tid, double *Sd,
                              Arena &ar, cudaStream_t s) {
  int v_lo = 0, v_hi = pr->n;   // the handle's v range (sox_set_v_range)
  v_range(h, pr->n, &v_lo, &v_hi);
  const int n = pr->n, N = pr->N, T = pr->n_tau, S = pr->n_spin, nO = n_omega;
  int ct = 1;
  kpoint_dynamic_bytes(h, n, N, T, nO, pr->nk, &ct);
  const int nk = pr->nk[0] * pr->nk[1] * pr->nk[2];
  const long long nn = (long long)n * n, Nn2 = (long long)N * nn, NN = (long long)N * N, Nn = (long long)N * n;
  const long long nk2 = (long long)nk * nk;
  const z *G = reinterpret_cast<const z *>(Gd);
  const z *X = reinterpret_cast<const z *>(Xd);
  const z *V = reinterpret_cast<const z *>(Vd);
  const z *Wd = reinterpret_cast<const z *>(Wdd);
  const z *Tf = reinterpret_cast<const z *>(Tfd);
  const z *Ti = reinterpret_cast<const z *>(Tid);
  z *Sig = reinterpret_cast<z *>(Sd);

  std::vector<int> add(nk * nk), sub(nk * nk);
  {
    auto idx = [&](int x, int y, int zz) {
      x = ((x % pr->nk[0]) + pr->nk[0]) % pr->nk[0];
      y = ((y % pr->nk[1]) + pr->nk[1]) % pr->nk[1];
      zz = ((zz % pr->nk[2]) + pr->nk[2]) % pr->nk[2];
      return (x * pr->nk[1] + y) * pr->nk[2] + zz;
    };
    for (int a = 0; a < nk; ++a)
      for (int b = 0; b < nk; ++b) {
        const int ax = a / (pr->nk[1] * pr->nk[2]), ay = (a / pr->nk[2]) % pr->nk[1], az = a % pr->nk[2];
        const int bx = b / (pr->nk[1] * pr->nk[2]), by = (b / pr->nk[2]) % pr->nk[1], bz = b % pr->nk[2];
        add[a * nk + b] = idx(ax + bx, ay + by, az + bz);
        sub[a * nk + b] = idx(ax - bx, ay - by, az - bz);
      }
  }
  int *d_add = ar.take<int>(nk2), *d_sub = ar.take<int>(nk2);
  z *Y = ar.take<z>(nk2 * Nn2), *M2 = ar.take<z>(nk2 * Nn2);
  z *GWt = ar.take<z>((size_t)nk * T * Nn), *GR = ar.take<z>((size_t)nk * T * Nn);
  z *GG = ar.take<z>((size_t)nk * T * Nn);
  z *GGw = ar.take<z>((size_t)nk * nO * Nn), *Aw = ar.take<z>((size_t)nk * nO * Nn);
  z *A = ar.take<z>((size_t)nk2 * T * Nn);
  z *D = ar.take<z>((size_t)T * nk * NN), *T1 = ar.take<z>((size_t)2 * nk * Nn);
  long long *wA = ar.take<long long>((size_t)nk2 * nO), *wB = ar.take<long long>((size_t)nk * nO);
  z *Bc = ar.take<z>((size_t)nk2 * ct * NN), *Cc = ar.take<z>((size_t)nk2 * ct * NN);
  long long *oA = ar.take<long long>(nk2 * ct), *oB = ar.take<long long>(nk2 * ct);
  long long *oC = ar.take<long long>(nk2 * ct), *oD = ar.take<long long>(nk2 * ct);
  if (!oD) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  SOX_CUDA_TRY(cudaMemcpyAsync(d_add, add.data(), 4 * nk2, cudaMemcpyHostToDevice, s));
  SOX_CUDA_TRY(cudaMemcpyAsync(d_sub, sub.data(), 4 * nk2, cudaMemcpyHostToDevice, s));
  {  // offsets of the W_d product: batch b = ks * nO + m; A = W_d[q1][m] (q1 added per launch), B/C = [ks][m]
    std::vector<long long> ha(nk2 * nO), hb(nk * nO);
    for (int q = 0; q < nk; ++q)
      for (int ks = 0; ks < nk; ++ks)
        for (int m = 0; m < nO; ++m) ha[((long long)q * nk + ks) * nO + m] = ((long long)q * nO + m) * NN;
    for (int ks = 0; ks < nk; ++ks)
      for (int m = 0; m < nO; ++m) hb[(long long)ks * nO + m] = ((long long)ks * nO + m) * Nn;
    SOX_CUDA_TRY(cudaMemcpyAsync(wA, ha.data(), 8 * ha.size(), cudaMemcpyHostToDevice, s));
    SOX_CUDA_TRY(cudaMemcpyAsync(wB, hb.data(), 8 * hb.size(), cudaMemcpyHostToDevice, s));
  }
  ProfScope ps(h, "kpoint_dynamic_f64", s, 0);
  long long launches = 0;
  // bare mixed tensors M2[q][k'] for C
  k_kpair_products<<<grid1(nk2 * Nn2), 256, 0, s>>>(X, d_sub, nk, N, n, Y);
  for (int q = 0; q < nk; ++q) {
    ZGemm g = zg();
    g.M = N; g.Nc = (int)nn; g.K = N; g.batch = nk;
    g.A = V + (long long)q * NN; g.ai = N; g.ak = 1;
    g.B = Y + (long long)q * nk * Nn2; g.sB = Nn2; g.bk = nn; g.bj = 1;
    g.C = M2 + (long long)q * nk * Nn2; g.sC = Nn2; g.ci = nn; g.cj = 1;
    zgemm(g, s);
  }
  launches += 1 + nk;
  std::vector<long long> hA(nk2 * ct), hB(nk2 * ct), hC(nk2 * ct), hD(nk2 * ct);
  const double inv_nk2 = 1.0 / ((double)nk * nk);
  for (int sp = 0; sp < S; ++sp) {
    const z *Gs = G + (long long)sp * nk * T * nn;
    for (int k = 0; k < nk; ++k) {  // GWt[k][j][Q][u], GR[k][j][Q][v] for every tau
      ZGemm g = zg();
      g.M = N; g.Nc = n; g.K = n; g.batch = T;
      g.A = X + (long long)k * Nn; g.ai = n; g.ak = 1; g.conjA = 1;
      g.B = Gs + (long long)k * T * nn; g.sB = nn; g.bk = 1; g.bj = n;
      g.C = GWt + (long long)k * T * Nn; g.sC = Nn; g.ci = n; g.cj = 1;
      zgemm(g, s);
      ZGemm r = g;
      r.conjA = 0; r.bk = n; r.bj = 1; r.C = GR + (long long)k * T * Nn;
      zgemm(r, s);
      launches += 2;
    }
    SOX_CUDA_TRY(cudaMemsetAsync(D, 0, 16 * (size_t)T * nk * NN, s));
    for (int v = v_lo; v < v_hi; ++v) {   // the handle's v range (sox_set_v_range)
      for (int q1 = 0; q1 < nk; ++q1) {
        k_gg_k<<<grid1((long long)nk * T * Nn), 256, 0, s>>>(GWt, GR, d_sub, nk, q1, T, N, n, v, GG);
        ZGemm f = zg();  // GGw[ks][m] = sum_j T_fwd[m][j] GG[ks][j]
        f.M = nO; f.Nc = (int)Nn; f.K = T; f.batch = nk;
        f.A = Tf; f.ai = T; f.ak = 1;
        f.B = GG; f.sB = (long long)T * Nn; f.bk = Nn; f.bj = 1;
        f.C = GGw; f.sC = (long long)nO * Nn; f.ci = Nn; f.cj = 1;
        zgemm(f, s);
        ZGemm w = zg();  // Aw[ks][m][P][u] = sum_Q W_d[q1][m][P][Q] GGw[ks][m][Q][u]
        w.M = N; w.Nc = n; w.K = N; w.batch = nk * nO;
        w.A = Wd; w.offA = wA + (long long)q1 * nk * nO; w.ai = N; w.ak = 1;
        w.B = GGw; w.offB = wB; w.bk = n; w.bj = 1;
        w.C = Aw; w.offC = wB; w.ci = n; w.cj = 1;
        zgemm(w, s);
        ZGemm iv = zg();  // A[(q1, ks)][i] = sum_m T_inv[i][m] Aw[ks][m]
        iv.M = T; iv.Nc = (int)Nn; iv.K = nO; iv.batch = nk;
        iv.A = Ti; iv.ai = nO; iv.ak = 1;
        iv.B = Aw; iv.sB = (long long)nO * Nn; iv.bk = Nn; iv.bj = 1;
        iv.C = A + (long long)q1 * nk * T * Nn; iv.sC = (long long)T * Nn; iv.ci = Nn; iv.cj = 1;
        zgemm(iv, s);
        launches += 4;
      }
      for (int i0 = 0; i0 < T; i0 += ct) {
        const int cc = std::min(ct, T - i0);
        for (int q = 0; q < nk; ++q)
          for (int kk = 0; kk < nk; ++kk)
            for (int il = 0; il < cc; ++il) {
              const long long b = ((long long)q * nk + kk) * cc + il;
              hA[b] = (((long long)q * nk + kk) * T + i0 + il) * Nn;       // A[(q1, ks)][i]
              hB[b] = (long long)sub[kk * nk + q] * Nn;                    // X[k_u]
              hC[b] = ((long long)kk * T + i0 + il) * Nn;                  // GWt[k_w][i]
              hD[b] = ((long long)q * nk + kk) * Nn2 + (long long)v * n;   // M2[(q2, k_w)][.][v][.]
            }
        const long long nb = nk2 * cc;
        SOX_CUDA_TRY(cudaMemcpyAsync(oA, hA.data(), 8 * nb, cudaMemcpyHostToDevice, s));
        SOX_CUDA_TRY(cudaMemcpyAsync(oB, hB.data(), 8 * nb, cudaMemcpyHostToDevice, s));
        SOX_CUDA_TRY(cudaMemcpyAsync(oC, hC.data(), 8 * nb, cudaMemcpyHostToDevice, s));
        SOX_CUDA_TRY(cudaMemcpyAsync(oD, hD.data(), 8 * nb, cudaMemcpyHostToDevice, s));
        ZGemm gb = zg();  // B[b][P][R] = sum_u A[b][P][u] X[k_u][R][u]
        gb.M = N; gb.Nc = N; gb.K = n; gb.batch = (int)nb;
        gb.A = A; gb.offA = oA; gb.ai = n; gb.ak = 1;
        gb.B = X; gb.offB = oB; gb.bk = 1; gb.bj = n;
        gb.C = Bc; gb.sC = NN; gb.ci = N; gb.cj = 1;
        zgemm(gb, s);
        ZGemm gc = zg();  // C[b][P][R] = sum_w GWt[k_w][i][P][w] M2[(q2, k_w)][R][v][w]
        gc.M = N; gc.Nc = N; gc.K = n; gc.batch = (int)nb;
        gc.A = GWt; gc.offA = oC; gc.ai = n; gc.ak = 1;
        gc.B = M2; gc.offB = oD; gc.bk = 1; gc.bj = nn;
        gc.C = Cc; gc.sC = NN; gc.ci = N; gc.cj = 1;
        zgemm(gc, s);
        dim3 grid((N + 31) / 32, (N + 7) / 8, nk * cc);
        k_kpoint_D_tau<<<grid, dim3(32, 8), 0, s>>>(Bc, Cc, d_add, d_sub, nk, N, cc, i0, D);
        launches += 3;
      }
    }
    for (int i = 0; i < T; ++i) {  // Sigma^k(tau_i) += -1/N_k^2 X_k^H D[i][k]^T X_k
      ZGemm t = zg();
      t.M = N; t.Nc = n; t.K = N; t.batch = nk;
      t.A = D + (long long)i * nk * NN; t.sA = NN; t.ai = 1; t.ak = N;
      t.B = X; t.sB = Nn; t.bk = n; t.bj = 1;
      t.C = T1; t.sC = Nn; t.ci = n; t.cj = 1;
      zgemm(t, s);
      ZGemm o = zg();
      o.M = n; o.Nc = n; o.K = N; o.batch = nk;
      o.A = X; o.sA = Nn; o.ai = 1; o.ak = n; o.conjA = 1;
      o.B = T1; o.sB = Nn; o.bk = n; o.bj = 1;
      o.C = Sig + ((long long)sp * nk * T + i) * nn; o.sC = (long long)T * nn; o.ci = n; o.cj = 1;
      o.alpha = -inv_nk2; o.beta = 1.0;
      zgemm(o, s);
      launches += 2;
    }
  }
  h->launches += launches;
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

// ---------------------------------------------------------------------------
// Split-precision forms (SOX_PREC_F16X2): every contraction of the chain as a
// complex FP16-pair GEMM on the tensor cores (ctc.cu), FP32 results; the
// projections, the D accumulation over v and the back-projection stay FP64.
// ---------------------------------------------------------------------------
namespace {

struct KTc {
  int nk, n, N, T, S;
  long long nk2, nn, Nn, NN, Nn2;
  int ldN;    // complex row length of B, C and D (N rounded up to even)
};

KTc ktc_geom(const sox_problem *p) {
  KTc g;
  g.nk = p->nk[0] * p->nk[1] * p->nk[2];
  g.n = p->n;
  g.N = p->N;
  g.T = p->n_tau;
  g.S = p->n_spin;
  g.nk2 = (long long)g.nk * g.nk;
  g.nn = (long long)g.n * g.n;
  g.Nn = (long long)g.N * g.n;
  g.NN = (long long)g.N * g.N;
  g.Nn2 = g.Nn * g.n;
  g.ldN = g.N + (g.N & 1);
  return g;
}

// device tables: add, sub (n_k x n_k), kk[pair] = pair % n_k, ku[pair] = sub[pair % n_k][pair / n_k]
struct KTables {
  int *add = nullptr, *sub = nullptr, *kk = nullptr, *ku = nullptr, *qq = nullptr;
  std::vector<int> h_add, h_sub;
};

Status ktc_tables(const sox_problem *pr, const KTc &g, Arena &ar, cudaStream_t s, KTables *t) {
  mesh_tables(pr, t->h_add, t->h_sub);
  std::vector<int> kk(g.nk2), ku(g.nk2), qq(g.nk2);
  for (long long pr_ = 0; pr_ < g.nk2; ++pr_) {
    const int ks = (int)(pr_ % g.nk), q = (int)(pr_ / g.nk);
    kk[pr_] = ks;
    qq[pr_] = q;
    ku[pr_] = t->h_sub[(size_t)ks * g.nk + q];
  }
  t->add = ar.take<int>(g.nk2);
  t->sub = ar.take<int>(g.nk2);
  t->kk = ar.take<int>(g.nk2);
  t->ku = ar.take<int>(g.nk2);
  t->qq = ar.take<int>(g.nk2);
  if (!t->qq) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  SOX_CUDA_TRY(cudaMemcpyAsync(t->add, t->h_add.data(), 4 * g.nk2, cudaMemcpyHostToDevice, s));
  SOX_CUDA_TRY(cudaMemcpyAsync(t->sub, t->h_sub.data(), 4 * g.nk2, cudaMemcpyHostToDevice, s));
  SOX_CUDA_TRY(cudaMemcpyAsync(t->kk, kk.data(), 4 * g.nk2, cudaMemcpyHostToDevice, s));
  SOX_CUDA_TRY(cudaMemcpyAsync(t->ku, ku.data(), 4 * g.nk2, cudaMemcpyHostToDevice, s));
  SOX_CUDA_TRY(cudaMemcpyAsync(t->qq, qq.data(), 4 * g.nk2, cudaMemcpyHostToDevice, s));
  return Status::ok();
}

size_t tables_bytes(const KTc &g) { return 5 * aligned_bytes(g.nk2, 4); }

long long nnpad_of(const KTc &g) { return g.nn + (g.nn & 1); }

// scratch of mixed_tc (released after the call)
size_t mixed_tc_scratch(const KTc &g) {
  return csplit_bytes(g.nk, g.N, g.N) + csplit_bytes((int)g.nk2, (int)(2 * g.nn), g.N);
}
size_t mixed_tc_bytes(const KTc &g) { return aligned_bytes((size_t)g.nk2 * g.N * nnpad_of(g), 8); }

// Mixed tensor on the tensor cores, FP32 complex [pair][P][(a,b)] with row length nnpad:
//   M^{q,k'}[P][(a,b)] = sum_Q U^q[P][Q] conj(X^{k'-q}[Q][a]) X^{k'}[Q][b]
Status mixed_tc(sox_handle h, const z *X, const z *U, const KTables &tb, const KTc &g, Arena scratch, float *M,
                cudaStream_t s) {
  CSplit Us = csplit_take(scratch, g.nk, g.N, g.N);
  CSplit Ys = csplit_take(scratch, (int)g.nk2, (int)(2 * g.nn), g.N);
  if (!Ys.hi) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  csplit_a(U, false, g.NN, g.N, 0, 0, 1, g.nk, g.N, g.N, Us, s);
  csplit_pairs(reinterpret_cast<const double *>(X), tb.sub, g.nk, g.N, g.n, Ys, s);
  h->launches += 2;
  const long long ld = nnpad_of(g);
  return cgemm_tc(h, Us, Ys, (int)g.nk2, tb.qq, nullptr, 1.f, M, 2 * ld, 2 * g.N * ld, s);
}

// B rows (P,q) of the first mixed tensor, K = s
void split_m1_tc(const float *M, const KTc &g, const CSplit &M1s, cudaStream_t s) {
  const long long ld = nnpad_of(g);
  csplit_b(M, true, g.N * ld, ld, g.n, g.n, 1, (int)g.nk2, (int)g.Nn, g.n, false, false, M1s, s);
}

void split_m2_tc(const float *M, const KTc &g, const std::vector<CSplit> &M2s, cudaStream_t s) {
  const long long ld = nnpad_of(g);
  for (int v = 0; v < g.n; ++v)
    csplit_b(reinterpret_cast<const float2 *>(M) + (long long)v * g.n, true, g.N * ld, ld, 0, 0, 1, (int)g.nk2, g.N,
             g.n, false, false, M2s[v], s);
}

// Sigma^k(tau_i) (+)= alpha X_k^H D[k]^T X_k for every k (D FP64 [k][N][ldN])
void backproject_k(const z *D, const z *X, const KTc &g, z *T1, z *Sig_i, long long sS, double alpha, double beta,
                   cudaStream_t s) {
  ZGemm t = zg();
  t.M = g.N; t.Nc = g.n; t.K = g.N; t.batch = g.nk;
  t.A = D; t.sA = (long long)g.N * g.ldN; t.ai = 1; t.ak = g.ldN;
  t.B = X; t.sB = g.Nn; t.bk = g.n; t.bj = 1;
  t.C = T1; t.sC = g.Nn; t.ci = g.n; t.cj = 1;
  zgemm(t, s);
  ZGemm o = zg();
  o.M = g.n; o.Nc = g.n; o.K = g.N; o.batch = g.nk;
  o.A = X; o.sA = g.Nn; o.ai = 1; o.ak = g.n; o.conjA = 1;
  o.B = T1; o.sB = g.Nn; o.bk = g.n; o.bj = 1;
  o.C = Sig_i; o.sC = sS; o.ci = g.n; o.cj = 1;
  o.alpha = alpha; o.beta = beta;
  zgemm(o, s);
}

}  // namespace

size_t kpoint_tc_bytes(sox_handle, const sox_problem *p, bool two) {
  const KTc g = ktc_geom(p);
  size_t b = tables_bytes(g) + mixed_tc_bytes(g) * (two ? 2 : 1) + mixed_tc_scratch(g);
  const long long ldNn = g.Nn + (g.Nn & 1);
  b += csplit_bytes((int)g.nk2, (int)(2 * g.Nn), g.n) + (size_t)g.n * csplit_bytes((int)g.nk2, 2 * g.N, g.n);
  b += 2 * aligned_bytes(g.nk * g.Nn, 16);
  b += csplit_bytes(g.nk, 2 * g.N, g.n) + csplit_bytes(g.nk, g.N, g.n) + csplit_bytes(g.nk, g.n, g.n);
  b += aligned_bytes(g.nk2 * g.n * ldNn, 8) + csplit_bytes((int)g.nk2, g.N, g.n);
  b += 2 * aligned_bytes(g.nk2 * g.N * g.ldN, 8);
  b += aligned_bytes((size_t)g.nk * g.N * g.ldN, 16) + aligned_bytes(g.nk * g.Nn, 16);
  return b + (1 << 20);
}

Status kpoint_sigma_tc(sox_handle h, const sox_problem *pr, const double *Gd, const double *Xd, const double *U1d,
                       const double *U2d, double *Sd, Arena &ar, cudaStream_t s) {
  int v_lo = 0, v_hi = pr->n;   // the handle's v range (sox_set_v_range)
  v_range(h, pr->n, &v_lo, &v_hi);
  const KTc g = ktc_geom(pr);
  const bool two = (U1d != U2d);
  const z *G = reinterpret_cast<const z *>(Gd);
  const z *X = reinterpret_cast<const z *>(Xd);
  const z *U1 = reinterpret_cast<const z *>(U1d);
  const z *U2 = reinterpret_cast<const z *>(U2d);
  z *Sig = reinterpret_cast<z *>(Sd);
  KTables tb;
  SOX_TRY(ktc_tables(pr, g, ar, s, &tb));
  const size_t mfl = 2 * (size_t)g.nk2 * g.N * nnpad_of(g);
  float *M1 = ar.take<float>(mfl);
  float *M2 = two ? ar.take<float>(mfl) : M1;
  const long long ldNn = g.Nn + (g.Nn & 1);
  CSplit M1s = csplit_take(ar, (int)g.nk2, (int)(2 * g.Nn), g.n);
  std::vector<CSplit> M2s(g.n);
  for (int v = 0; v < g.n; ++v) M2s[v] = csplit_take(ar, (int)g.nk2, 2 * g.N, g.n);
  z *GR = ar.take<z>(g.nk * g.Nn), *GWt = ar.take<z>(g.nk * g.Nn);
  CSplit GRs = csplit_take(ar, g.nk, 2 * g.N, g.n), GWts = csplit_take(ar, g.nk, g.N, g.n);
  CSplit Gms = csplit_take(ar, g.nk, g.n, g.n);
  float *Aall = ar.take<float>(2 * g.nk2 * g.n * ldNn);
  CSplit As = csplit_take(ar, (int)g.nk2, g.N, g.n);
  float *Ball = ar.take<float>(2 * g.nk2 * g.N * g.ldN), *Call = ar.take<float>(2 * g.nk2 * g.N * g.ldN);
  z *D = ar.take<z>((size_t)g.nk * g.N * g.ldN), *T1 = ar.take<z>(g.nk * g.Nn);
  if (!T1 || !As.hi || !M1s.hi || !M2s.back().hi || !Gms.hi)
    return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  ProfScope ps(h, "kpoint_tc", s, 0);
  SOX_CUDA_TRY(cudaMemsetAsync(Ball, 0, 8 * g.nk2 * g.N * g.ldN, s));   // pad columns stay zero
  SOX_CUDA_TRY(cudaMemsetAsync(Call, 0, 8 * g.nk2 * g.N * g.ldN, s));
  SOX_TRY(mixed_tc(h, X, U1, tb, g, ar, M1, s));
  if (two) SOX_TRY(mixed_tc(h, X, U2, tb, g, ar, M2, s));
  split_m1_tc(M1, g, M1s, s);
  split_m2_tc(M2, g, M2s, s);
  long long launches = 1 + g.n;
  const double inv_nk2 = 1.0 / (double)g.nk2;
  for (int sp = 0; sp < g.S; ++sp) {
    const z *Gs = G + (long long)sp * g.nk * g.T * g.nn;
    for (int j = 0; j < g.T; ++j) {
      {  // FP64 projections at tau_j for every k
        ZGemm p = zg();
        p.M = g.N; p.Nc = g.n; p.K = g.n; p.batch = g.nk;
        p.A = X; p.sA = g.Nn; p.ai = g.n; p.ak = 1;
        p.B = Gs + (long long)j * g.nn; p.sB = (long long)g.T * g.nn; p.bk = g.n; p.bj = 1;
        p.C = GR; p.sC = g.Nn; p.ci = g.n; p.cj = 1;
        zgemm(p, s);
        ZGemm w = p;
        w.conjA = 1; w.bk = 1; w.bj = g.n; w.C = GWt;
        zgemm(w, s);
      }
      csplit_b(GR, false, g.Nn, g.n, 0, 0, 1, g.nk, g.N, g.n, false, false, GRs, s);
      csplit_a(GWt, false, g.Nn, g.n, 0, 0, 1, g.nk, g.N, g.n, GWts, s);
      // A rows v of G(-tau_j)^T: element (v, s) = G^k(tau_{T-1-j})[s][v]; the sign goes into alpha
      csplit_a(Gs + (long long)(g.T - 1 - j) * g.nn, false, (long long)g.T * g.nn, 1, 0, 0, g.n, g.nk, g.n, g.n, Gms,
               s);
      // A^{q1,ks}[v][(P,q)] = -sum_s G^{ks}(tau_{T-1-j})[s][v] M1[(P,q)][s]   ((P,q) contiguous per v)
      SOX_TRY(cgemm_tc(h, Gms, M1s, (int)g.nk2, tb.kk, nullptr, -1.f, Aall, 2 * ldNn, 2LL * g.n * ldNn, s));
      SOX_CUDA_TRY(cudaMemsetAsync(D, 0, 16 * (size_t)g.nk * g.N * g.ldN, s));
      launches += 5;
      for (int v = v_lo; v < v_hi; ++v) {   // the handle's v range (sox_set_v_range)
        csplit_a(reinterpret_cast<const float2 *>(Aall) + (long long)v * ldNn, true, g.n * ldNn, g.n, 0, 0, 1,
                 (int)g.nk2, g.N, g.n, As, s);
        {
          ProfScope pb(h, "kpoint_bc", s, 0);
          // B^{q1,ks}_v[P][R] = sum_q A[v][P][q] GR^{ks-q1}[R][q]
          SOX_TRY(cgemm_tc(h, As, GRs, (int)g.nk2, nullptr, tb.ku, 1.f, Ball, 2LL * g.ldN, 2LL * g.N * g.ldN, s));
          // C^{q2,kw}_v[P][R] = sum_w GWt^{kw}[P][w] M2^{q2,kw}[R][v][w]
          SOX_TRY(
              cgemm_tc(h, GWts, M2s[v], (int)g.nk2, tb.kk, nullptr, 1.f, Call, 2LL * g.ldN, 2LL * g.N * g.ldN, s));
        }
        {
          ProfScope pd(h, "kpoint_D", s, 0);
          SOX_TRY(kpoint_D_f32(Ball, Call, (long long)g.N * g.ldN, 0, tb.add, tb.sub, pr->nk, (long long)g.N * g.ldN,
                               1, 0, 0, reinterpret_cast<double *>(D), s));
        }
        launches += 2;
      }
      backproject_k(D, X, g, T1, Sig + ((long long)sp * g.nk * g.T + j) * g.nn, (long long)g.T * g.nn, -inv_nk2, 0.0,
                    s);
      launches += 4;
    }
  }
  h->launches += launches;
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

namespace {

struct KDynTc {
  KTc g;
  int nO, ct, upad;
  long long ldNn;   // complex row length of GG(i Omega) and of A(tau) rows: N n rounded up to even
};

KDynTc kdyn_geom(sox_handle h, const sox_problem *p, int nO, size_t *fixed_out, size_t *per_t_out) {
  KDynTc d;
  d.g = ktc_geom(p);
  const KTc &g = d.g;
  d.nO = nO;
  d.upad = g.n + (g.n & 1);
  d.ldNn = g.Nn + (g.Nn & 1);
  size_t f = tables_bytes(g) + aligned_bytes((size_t)g.nk2 * nO, 4);
  f += mixed_tc_bytes(g) + mixed_tc_scratch(g);                                 // M2 (FP32) and its scratch
  f += (size_t)g.n * csplit_bytes((int)g.nk2, 2 * g.N, g.n);                    // M2 split per v
  f += csplit_bytes(g.nk, 2 * g.N, g.n);                                        // X split
  f += csplit_bytes(g.nk * nO, g.N, g.N);                                       // W_d split
  f += csplit_bytes(1, nO, g.T) + csplit_bytes(1, g.T, nO);                     // transforms
  f += 3 * aligned_bytes((size_t)g.nk * g.T * g.Nn, 16);                        // GR, GWt, GG (FP64)
  f += csplit_bytes(g.nk, g.T * g.N, g.n);                                      // GWt split, all tau
  f += csplit_bytes(g.nk, (int)(2 * g.Nn), g.T);                                // GG split
  f += aligned_bytes((size_t)g.nk * nO * d.ldNn, 8);                            // GG(i Omega)
  f += csplit_bytes(g.nk * nO, 2 * g.n, g.N);                                   // its split
  f += aligned_bytes((size_t)g.nk * nO * g.N * d.upad, 8);                      // W_d GG
  f += csplit_bytes(g.nk, (int)(2 * g.Nn), nO);                                 // its split
  f += aligned_bytes((size_t)g.nk2 * g.T * d.ldNn, 8);                          // A(tau), all pairs
  f += aligned_bytes((size_t)g.T * g.nk * g.N * g.ldN, 16);                     // D for every tau
  f += aligned_bytes(g.nk * g.Nn, 16) + (1 << 20);
  const size_t per_t = csplit_bytes((int)g.nk2, g.N, g.n) + 2 * aligned_bytes(g.nk2 * g.N * g.ldN, 8);
  const size_t budget = chunk_budget(h, size_t(24) << 30);
  long long ct = budget > f ? (long long)((budget - f) / per_t) : 1;
  d.ct = (int)std::max<long long>(1, std::min<long long>(ct, g.T));
  if (fixed_out) *fixed_out = f;
  if (per_t_out) *per_t_out = per_t;
  return d;
}

}  // namespace

size_t kpoint_dynamic_tc_bytes(sox_handle h, const sox_problem *p, int n_omega) {
  size_t f = 0, per_t = 0;
  const KDynTc d = kdyn_geom(h, p, n_omega, &f, &per_t);
  return f + per_t * d.ct + (1 << 20);
}

Status kpoint_dynamic_tc(sox_handle h, const sox_problem *pr, int n_omega, const double *Gd, const double *Xd,
                         const double *Vd, const double *Wdd, const double *Tfd, const double *Tid, double *Sd,
                         Arena &ar, cudaStream_t s) {
  int v_lo = 0, v_hi = pr->n;   // the handle's v range (sox_set_v_range)
  v_range(h, pr->n, &v_lo, &v_hi);
  const KDynTc d = kdyn_geom(h, pr, n_omega, nullptr, nullptr);
  const KTc &g = d.g;
  const int nO = d.nO, T = g.T, n = g.n, N = g.N, nk = g.nk;
  const z *G = reinterpret_cast<const z *>(Gd);
  const z *X = reinterpret_cast<const z *>(Xd);
  const z *V = reinterpret_cast<const z *>(Vd);
  z *Sig = reinterpret_cast<z *>(Sd);
  KTables tb;
  SOX_TRY(ktc_tables(pr, g, ar, s, &tb));
  int *widx = ar.take<int>((size_t)g.nk2 * nO);
  float *M2 = ar.take<float>(2 * (size_t)g.nk2 * N * nnpad_of(g));
  std::vector<CSplit> M2s(n);
  for (int v = 0; v < n; ++v) M2s[v] = csplit_take(ar, (int)g.nk2, 2 * N, n);
  CSplit Xs = csplit_take(ar, nk, 2 * N, n);
  CSplit Wds = csplit_take(ar, nk * nO, N, N);
  CSplit Tfs = csplit_take(ar, 1, nO, T), Tis = csplit_take(ar, 1, T, nO);
  z *GR = ar.take<z>((size_t)nk * T * g.Nn), *GWt = ar.take<z>((size_t)nk * T * g.Nn);
  z *GG = ar.take<z>((size_t)nk * T * g.Nn);
  CSplit GWts = csplit_take(ar, nk, T * N, n);
  CSplit GGs = csplit_take(ar, nk, (int)(2 * g.Nn), T);
  float *GGw = ar.take<float>(2 * (size_t)nk * nO * d.ldNn);
  CSplit GGws = csplit_take(ar, nk * nO, 2 * n, N);
  float *Aw = ar.take<float>(2 * (size_t)nk * nO * N * d.upad);
  CSplit Aws = csplit_take(ar, nk, (int)(2 * g.Nn), nO);
  float *Adyn = ar.take<float>(2 * (size_t)g.nk2 * T * d.ldNn);
  z *Dall = ar.take<z>((size_t)T * nk * N * g.ldN), *T1 = ar.take<z>(g.nk * g.Nn);
  CSplit As = csplit_take(ar, (int)g.nk2, d.ct * N, n);
  float *Ball = ar.take<float>(2 * (size_t)g.nk2 * d.ct * N * g.ldN);
  float *Call = ar.take<float>(2 * (size_t)g.nk2 * d.ct * N * g.ldN);
  if (!Call || !As.hi || !Aws.hi || !GGws.hi || !GWts.hi || !Tis.hi || !M2s.back().hi)
    return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  {
    std::vector<int> hw((size_t)g.nk2 * nO);
    for (int q = 0; q < nk; ++q)
      for (int ks = 0; ks < nk; ++ks)
        for (int m = 0; m < nO; ++m) hw[((size_t)q * nk + ks) * nO + m] = q * nO + m;
    SOX_CUDA_TRY(cudaMemcpyAsync(widx, hw.data(), 4 * hw.size(), cudaMemcpyHostToDevice, s));
  }
  ProfScope ps(h, "kpoint_dynamic_tc", s, 0);
  long long launches = 0;
  SOX_CUDA_TRY(cudaMemsetAsync(Ball, 0, 8 * (size_t)g.nk2 * d.ct * N * g.ldN, s));
  SOX_CUDA_TRY(cudaMemsetAsync(Call, 0, 8 * (size_t)g.nk2 * d.ct * N * g.ldN, s));
  SOX_TRY(mixed_tc(h, X, V, tb, g, ar, M2, s));
  split_m2_tc(M2, g, M2s, s);
  csplit_b(X, false, g.Nn, n, 0, 0, 1, nk, N, n, false, false, Xs, s);
  csplit_a(Wdd, false, g.NN, N, 0, 0, 1, nk * nO, N, N, Wds, s);
  csplit_a(Tfd, false, 0, T, 0, 0, 1, 1, nO, T, Tfs, s);
  csplit_a(Tid, false, 0, nO, 0, 0, 1, 1, T, nO, Tis, s);
  launches += n + 4;
  const double inv_nk2 = 1.0 / (double)g.nk2;
  for (int sp = 0; sp < g.S; ++sp) {
    const z *Gs = G + (long long)sp * nk * T * g.nn;
    for (int k = 0; k < nk; ++k) {  // GWt[k][j][Q][u], GR[k][j][Q][v] for every tau, FP64
      ZGemm p = zg();
      p.M = N; p.Nc = n; p.K = n; p.batch = T;
      p.A = X + (long long)k * g.Nn; p.ai = n; p.ak = 1; p.conjA = 1;
      p.B = Gs + (long long)k * T * g.nn; p.sB = g.nn; p.bk = 1; p.bj = n;
      p.C = GWt + (long long)k * T * g.Nn; p.sC = g.Nn; p.ci = n; p.cj = 1;
      zgemm(p, s);
      ZGemm r = p;
      r.conjA = 0; r.bk = n; r.bj = 1; r.C = GR + (long long)k * T * g.Nn;
      zgemm(r, s);
      launches += 2;
    }
    // rows (tau_i, P) of GWt^k, K = w
    csplit_a(GWt, false, (long long)T * g.Nn, n, 0, 0, 1, nk, T * N, n, GWts, s);
    SOX_CUDA_TRY(cudaMemsetAsync(Dall, 0, 16 * (size_t)T * nk * N * g.ldN, s));
    ++launches;
    for (int v = v_lo; v < v_hi; ++v) {   // the handle's v range (sox_set_v_range)
      for (int q1 = 0; q1 < nk; ++q1) {
        k_gg_k<<<grid1((long long)nk * T * g.Nn), 256, 0, s>>>(GWt, GR, tb.sub, nk, q1, T, N, n, v, GG);
        // B rows (Q,u) of GG^{ks}, K = tau_j
        csplit_b(GG, false, (long long)T * g.Nn, 1, 0, 0, g.Nn, nk, (int)g.Nn, T, false, false, GGs, s);
        // GG(i Omega_m)[ks][(Q,u)] = sum_j T_fwd[m][j] GG[ks][j][(Q,u)]
        SOX_TRY(cgemm_tc(h, Tfs, GGs, nk, nullptr, nullptr, 1.f, GGw, 2 * d.ldNn, 2LL * nO * d.ldNn, s));
        // B rows u of GG(i Omega_m)^{ks}, K = Q
        csplit_b(reinterpret_cast<const float2 *>(GGw), true, d.ldNn, 1, 0, 0, n, nk * nO, n, N, false, false, GGws,
                 s);
        // (W_d GG)[(ks,m)][P][u] = sum_Q W_d^{q1}(i Omega_m)[P][Q] GG(i Omega_m)[ks][Q][u]
        SOX_TRY(cgemm_tc(h, Wds, GGws, nk * nO, widx + (size_t)q1 * nk * nO, nullptr, 1.f, Aw, 2LL * d.upad,
                         2LL * N * d.upad, s));
        // B rows (P,u) of W_d GG, K = Omega_m
        csplit_b(reinterpret_cast<const float2 *>(Aw), true, (long long)nO * N * d.upad, d.upad, 1, n,
                 (long long)N * d.upad, nk, (int)g.Nn, nO, false, false, Aws, s);
        // A^{q1,ks}(tau_i)[(P,u)] = sum_m T_inv[i][m] (W_d GG)[ks][m][(P,u)]
        SOX_TRY(cgemm_tc(h, Tis, Aws, nk, nullptr, nullptr, 1.f, Adyn + 2 * (size_t)q1 * nk * T * d.ldNn,
                         2 * d.ldNn, 2LL * T * d.ldNn, s));
        launches += 4;
      }
      for (int i0 = 0; i0 < T; i0 += d.ct) {
        const int cc = std::min(d.ct, T - i0);
        CSplit Ac = As;
        Ac.rows = cc * N;
        // rows (il, P) of A^{pair}(tau_{i0+il}), K = u
        csplit_a(reinterpret_cast<const float2 *>(Adyn) + (size_t)i0 * d.ldNn, true, (long long)T * d.ldNn, d.ldNn, n,
                 N, 1, (int)g.nk2, cc * N, n, Ac, s);
        {
          ProfScope pb(h, "kpoint_bc", s, 0);
          // B^{q1,ks}(tau_i)[P][R] = sum_u A[P][u] X^{ks-q1}[R][u]
          SOX_TRY(cgemm_tc(h, Ac, Xs, (int)g.nk2, nullptr, tb.ku, 1.f, Ball, 2LL * g.ldN, 2LL * cc * N * g.ldN, s));
          // C^{q2,kw}(tau_i)[P][R] = sum_w GWt^{kw}(tau_i)[P][w] M2^{q2,kw}[R][v][w]
          SOX_TRY(cgemm_tc(h, GWts.view((long long)i0 * N, cc * N), M2s[v], (int)g.nk2, tb.kk, nullptr, 1.f, Call,
                           2LL * g.ldN, 2LL * cc * N * g.ldN, s));
        }
        {
          ProfScope pd(h, "kpoint_D", s, 0);
          SOX_TRY(kpoint_D_f32(Ball, Call, (long long)cc * N * g.ldN, (long long)N * g.ldN, tb.add, tb.sub, pr->nk,
                               (long long)N * g.ldN, cc, i0, (long long)nk * N * g.ldN,
                               reinterpret_cast<double *>(Dall), s));
        }
        launches += 2;
      }
    }
    for (int i = 0; i < T; ++i) {
      backproject_k(Dall + (size_t)i * nk * N * g.ldN, X, g, T1, Sig + ((long long)sp * nk * T + i) * g.nn,
                    (long long)T * g.nn, -inv_nk2, 1.0, s);
      launches += 2;
    }
  }
  h->launches += launches;
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}


// ===========================================================================
// RPA screened interaction on the transform's bosonic frequencies (the input of the
// dynamic path), for every transfer q of the mesh (a molecule is the mesh 1x1x1):
//   Pi^q(tau_j)_PQ = 1/N_k sum_k G^PQ_{k+q}(tau_j) G^QP_k(-tau_j),  G^PQ_k = X^k G^k X^k^H
//   Pi^q(i Omega_o) = sum_j T_fwd[o][j] Pi^q(tau_j)
//   W_d^q(i Omega_o) = (1 - V^q Pi^q(i Omega_o))^-1 V^q - V^q
// The k sum is a cyclic cross-correlation over the mesh: with A-hat(m) = sum_k w^{-m.k}
// A_k (one in-place DFT of the projections over k), its transform is the pointwise product
// A-hat_{tau_j}(m)[P][Q] A-hat_{tau_{T-1-j}}(-m)[Q][P] (G(-tau_j) = -G(tau_{T-1-j})), so
// the bubble of every q costs one pass over the projections and an inverse DFT over m.
// FP64 throughout; the solve is Gauss-Jordan with partial pivoting, batched over (q, o).
namespace {

constexpr int kMaxSide = 8;

__global__ void k_r2c(const double *src, z *dst, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = make_double2(src[e], 0.0);
}

// twiddles exp(sgn 2 pi i r / Nd), r < Nd (computed on the host)
struct MeshTw {
  double2 w[kMaxSide];
};

// in-place DFT along mesh dimension dim of buf[k][.] (k row-major over n1 x n2 x n3, k-th
// block at k * kstride, its first `inner` elements transformed):
// out[m] = sum_t exp(sgn 2 pi i m t / Nd) in[t]
__global__ void k_mesh_dft(z *buf, long long inner, long long kstride, int n1, int n2, int n3, int dim, MeshTw tw) {
  const int Nd = dim == 0 ? n1 : (dim == 1 ? n2 : n3);
  const long long sd = (dim == 0 ? (long long)n2 * n3 : (dim == 1 ? n3 : 1)) * kstride;
  const long long lines = (long long)(n1 * n2 * n3 / Nd) * inner;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < lines;
       g += (long long)gridDim.x * blockDim.x) {
    const long long e = g % inner;
    const int r = (int)(g / inner);
    int kb;
    if (dim == 0)
      kb = r;                                   // (c1, c2) with c0 = 0: r = c1 n3 + c2
    else if (dim == 1)
      kb = (r / n3) * n2 * n3 + (r % n3);       // (c0, c2)
    else
      kb = r * n3;                              // (c0, c1)
    z *base = buf + (long long)kb * kstride + e;
    z v[kMaxSide];
#pragma unroll
    for (int t = 0; t < kMaxSide; ++t)
      if (t < Nd) v[t] = base[t * sd];
#pragma unroll
    for (int m = 0; m < kMaxSide; ++m) {
      if (m >= Nd) break;
      z acc = v[0];
#pragma unroll
      for (int t = 1; t < kMaxSide; ++t) {
        if (t >= Nd) break;
        acc = zfma(tw.w[(m * t) % Nd], v[t], acc);
      }
      base[m * sd] = acc;
    }
  }
}

// H[m][o][P][Q] += alpha sum_j T_fwd[o][j] Ah[m][j][P][Q] Ah[negm[m]][T-1-j][Q][P] for the
// kBubF frequencies o of chunk blockIdx.z % n_chunks; 32 x 32 tiles, the transposed
// partner through shared memory
constexpr int kBubF = 4;
__global__ void __launch_bounds__(256) k_bubble_reduce(const z *Ah, const z *Tf, const int *negm, int N, int T, int nO,
                                                       int n_solve, int n_chunks, double alpha, z *H) {
  __shared__ z ta[32][33];
  __shared__ z tb[32][33];
  const int m = blockIdx.z / n_chunks, o0 = (blockIdx.z % n_chunks) * kBubF;
  const int P0 = blockIdx.y * 32, Q0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  const long long NN = (long long)N * N;
  const z *Am = Ah + (long long)m * T * NN, *Bm = Ah + (long long)negm[m] * T * NN;
  z acc[4][kBubF];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int f = 0; f < kBubF; ++f) acc[i][f] = make_double2(0.0, 0.0);
  for (int j = 0; j < T; ++j) {
    const z *Aj = Am + (long long)j * NN, *Bj = Bm + (long long)(T - 1 - j) * NN;
    for (int r = ty; r < 32; r += 8) {
      const int P = P0 + r, Q = Q0 + tx;
      ta[r][tx] = (P < N && Q < N) ? Aj[(long long)P * N + Q] : make_double2(0.0, 0.0);
      const int Qb = Q0 + r, Pb = P0 + tx;
      tb[r][tx] = (Qb < N && Pb < N) ? Bj[(long long)Qb * N + Pb] : make_double2(0.0, 0.0);   // tb[Q][P]
    }
    __syncthreads();
    z w[kBubF];
#pragma unroll
    for (int f = 0; f < kBubF; ++f) w[f] = (o0 + f < n_solve) ? Tf[(long long)(o0 + f) * T + j] : make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = ty + 8 * i;
      const z pr = zmul(ta[r][tx], tb[tx][r]);
#pragma unroll
      for (int f = 0; f < kBubF; ++f) acc[i][f] = zfma(w[f], pr, acc[i][f]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int P = P0 + ty + 8 * i, Q = Q0 + tx;
    if (P >= N || Q >= N) continue;
#pragma unroll
    for (int f = 0; f < kBubF; ++f) {
      if (o0 + f >= n_solve) break;
      z *h = H + ((long long)m * nO + o0 + f) * NN + (long long)P * N + Q;
      const z v = *h;
      *h = make_double2(v.x + alpha * acc[i][f].x, v.y + alpha * acc[i][f].y);
    }
  }
}

// molecules: Pi(i Omega) <- (Re Pi + Re Pi^T) / 2 in place, per frequency
__global__ void k_sym_real(z *Pi, int N, int nO) {
  const long long NN = (long long)N * N, total = NN * nO;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long o = g / NN, e = g % NN;
    const int P = (int)(e / N), Q = (int)(e % N);
    if (P > Q) continue;
    z *a = Pi + o * NN + (long long)P * N + Q, *b = Pi + o * NN + (long long)Q * N + P;
    const double s = 0.5 * (a->x + b->x);
    *a = make_double2(s, 0.0);
    *b = make_double2(s, 0.0);
  }
}

// Aug[b] = [I | V^{b / ns}] for every system b (ns systems per transfer), [N][2N]
__global__ void k_gj_init_c(const z *V, int N, int ns, int batch, z *Aug) {
  const long long NN = (long long)N * N, total = NN * batch;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long b = g / NN, e = g % NN;
    const int i = (int)(e / N), j = (int)(e % N);
    z *row = Aug + b * 2 * NN + (long long)i * 2 * N;
    row[j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    row[N + j] = V[(b / ns) * NN + e];
  }
}

// Gauss-Jordan step k of every system (one block each): the row of largest |a_ik|, i >= k,
// is swapped into row k and row k is divided by its pivot; info[1] is set for a zero column
__global__ void __launch_bounds__(256) k_gj_pivot_c(z *Aug, int N, int k, int *info) {
  __shared__ double best[256];
  __shared__ int bidx[256];
  const long long W = 2LL * N;
  z *A = Aug + (long long)blockIdx.x * N * W;
  double bv = -1.0;
  int bi = k;
  for (int i = k + threadIdx.x; i < N; i += blockDim.x) {
    const z a = A[(long long)i * W + k];
    const double m2 = a.x * a.x + a.y * a.y;
    if (m2 > bv) {
      bv = m2;
      bi = i;
    }
  }
  best[threadIdx.x] = bv;
  bidx[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double ov = best[threadIdx.x + o];
      const int oi = bidx[threadIdx.x + o];
      if (ov > best[threadIdx.x] || (ov == best[threadIdx.x] && oi < bidx[threadIdx.x])) {
        best[threadIdx.x] = ov;
        bidx[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (!(best[0] > 0.0)) {
    if (threadIdx.x == 0) atomicExch(&info[1], 1);
    return;
  }
  const int p = bidx[0];
  const z pv = A[(long long)p * W + k];
  const double d = pv.x * pv.x + pv.y * pv.y;
  const z inv = make_double2(pv.x / d, -pv.y / d);
  for (long long j = k + threadIdx.x; j < W; j += blockDim.x) {
    const z a = A[(long long)k * W + j];
    const z b = A[(long long)p * W + j];
    if (p != k) A[(long long)p * W + j] = a;
    A[(long long)k * W + j] = zmul(b, inv);
  }
}

// step k, part 2: column k eliminated from every other row (columns > k of both halves)
__global__ void k_gj_elim_c(z *Aug, int N, int k, const int *info) {
  if (info[1]) return;
  const long long W = 2LL * N;
  z *A = Aug + (long long)blockIdx.z * N * W;
  const int ncols = (int)(W - (k + 1));
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  const long long col = k + 1 + j;
  const z rk = A[(long long)k * W + col];
  for (int i = blockIdx.y; i < N; i += gridDim.y) {
    if (i == k) continue;
    const z f = A[(long long)i * W + k];
    z *c = A + (long long)i * W + col;
    *c = zfma(make_double2(-f.x, -f.y), rk, *c);
  }
}

// W_d[q][o] = right half of Aug[b] - V^q for system b = q ns + o (o < ns); molecules keep
// the real part
__global__ void k_gj_out(const z *Aug, const z *V, int N, int nO, int ns, int batch, int real_out, double *Wd) {
  const long long NN = (long long)N * N, total = NN * batch;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long b = g / NN, e = g % NN;
    const int i = (int)(e / N), j = (int)(e % N);
    const long long q = b / ns, out = (q * nO + b % ns) * NN + e;
    const z w = Aug[b * 2 * NN + (long long)i * 2 * N + N + j], v = V[q * NN + e];
    if (real_out)
      Wd[out] = w.x - v.x;
    else
      reinterpret_cast<z *>(Wd)[out] = make_double2(w.x - v.x, w.y - v.y);
  }
}

// W_d^q(-Omega) = W_d^q(Omega)^H: frequencies o >= ns from o' = nO - 1 - o < ns
__global__ void k_w_mirror(double *Wd, int N, int nO, int ns, int nq, int real_out) {
  const long long NN = (long long)N * N, per = (long long)(nO - ns) * NN, total = per * nq;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long q = g / per, r = g % per;
    const int o = ns + (int)(r / NN);
    const long long e = r % NN;
    const int i = (int)(e / N), j = (int)(e % N);
    const long long dst = (q * nO + o) * NN + e, src = (q * nO + (nO - 1 - o)) * NN + (long long)j * N + i;
    if (real_out) {
      Wd[dst] = Wd[src];
    } else {
      const z v = reinterpret_cast<const z *>(Wd)[src];
      reinterpret_cast<z *>(Wd)[dst] = make_double2(v.x, -v.y);
    }
  }
}

// out[0] = max |G|, out[1] = max |G_pq - conj(G_qp)| over count matrices n x n (as the bit
// patterns of non-negative doubles, which order like the values)
__global__ void k_herm_dev(const z *G, int n, long long count, unsigned long long *out) {
  const long long nn = (long long)n * n, total = nn * count;
  double m = 0.0, d = 0.0;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long c = g / nn, e = g % nn;
    const int p = (int)(e / n), q = (int)(e % n);
    const z a = G[g], b = G[c * nn + (long long)q * n + p];
    m = fmax(m, fmax(fabs(a.x), fabs(a.y)));
    d = fmax(d, fmax(fabs(a.x - b.x), fabs(a.y + b.y)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], (unsigned long long)__double_as_longlong(m));
    atomicMax(&out[1], (unsigned long long)__double_as_longlong(d));
  }
}

unsigned grid_of(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 1 << 20)); }

void mesh_dft(z *buf, long long inner, long long kstride, const int nk3[3], int sgn, cudaStream_t s) {
  for (int d = 0; d < 3; ++d) {
    if (nk3[d] == 1) continue;
    MeshTw tw{};
    for (int r = 0; r < nk3[d]; ++r) {
      const double a = 2.0 * 3.14159265358979323846 * r / nk3[d];
      tw.w[r] = make_double2(std::cos(a), sgn * std::sin(a));
    }
    const long long lines = (long long)(nk3[0] * nk3[1] * nk3[2] / nk3[d]) * inner;
    k_mesh_dft<<<grid_of(lines), 256, 0, s>>>(buf, inner, kstride, nk3[0], nk3[1], nk3[2], d, tw);
  }
}

}  // namespace

size_t w_dynamic_bytes(const sox_problem *p, int n_omega) {
  const size_t nk = (size_t)p->nk[0] * p->nk[1] * p->nk[2];
  const size_t N = p->N, n = p->n, T = p->n_tau, NN = N * N;
  size_t b = 0;
  if (p->dtype != SOX_COMPLEX128)   // complex copies of G, X, V
    b += aligned_bytes((size_t)p->n_spin * T * n * n, 16) + aligned_bytes(N * n, 16) + aligned_bytes(NN, 16);
  b += aligned_bytes(T * N * n, 16);                 // X^k G^k(tau)
  b += aligned_bytes(nk * T * NN, 16);               // projections, then their DFT over k
  b += aligned_bytes(nk * n_omega * NN, 16);         // the bubble per (m, o), then per (q, o)
  b += aligned_bytes(nk * n_omega * 2 * NN, 16);     // [1 - V Pi | V] per (q, o)
  b += aligned_bytes(nk, 4) + aligned_bytes(4, 4) + aligned_bytes(2, 8);
  return b + (1 << 20);
}

Status w_dynamic(sox_handle h, const sox_problem *p, int n_omega, const double *Gd, const double *Xd,
                 const double *Vd, const double *Tfd, double *Wd, Arena &ar, cudaStream_t s) {
  const int nk3[3] = {p->nk[0], p->nk[1], p->nk[2]};
  const int nk = nk3[0] * nk3[1] * nk3[2];
  if (nk3[0] > kMaxSide || nk3[1] > kMaxSide || nk3[2] > kMaxSide)
    return {SOX_ERR_SHAPE, "sox_w_dynamic: mesh sides above 8 are not supported"};
  const int N = p->N, n = p->n, T = p->n_tau, S = p->n_spin, nO = n_omega;
  const long long NN = (long long)N * N, nn = (long long)n * n;
  const bool real = p->dtype != SOX_COMPLEX128;
  const z *G = reinterpret_cast<const z *>(Gd), *X = reinterpret_cast<const z *>(Xd);
  const z *V = reinterpret_cast<const z *>(Vd);
  if (real) {
    z *Gc = ar.take<z>((size_t)S * T * nn), *Xc = ar.take<z>((size_t)N * n), *Vc = ar.take<z>((size_t)NN);
    if (!Vc) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
    k_r2c<<<grid_of((long long)S * T * nn), 256, 0, s>>>(Gd, Gc, (long long)S * T * nn);
    k_r2c<<<grid_of((long long)N * n), 256, 0, s>>>(Xd, Xc, (long long)N * n);
    k_r2c<<<grid_of(NN), 256, 0, s>>>(Vd, Vc, NN);
    G = Gc;
    X = Xc;
    V = Vc;
  }
  const z *Tf = reinterpret_cast<const z *>(Tfd);
  z *GR = ar.take<z>((size_t)T * N * n), *Ah = ar.take<z>((size_t)nk * T * NN);
  z *H = ar.take<z>((size_t)nk * nO * NN), *Aug = ar.take<z>((size_t)nk * nO * 2 * NN);
  int *negm = ar.take<int>(nk), *info = ar.take<int>(4);
  unsigned long long *hdev = ar.take<unsigned long long>(2);
  if (!hdev) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  std::vector<int> h_neg(nk);
  for (int m = 0; m < nk; ++m) {
    const int a = m / (nk3[1] * nk3[2]), b = (m / nk3[2]) % nk3[1], c = m % nk3[2];
    h_neg[m] = (((nk3[0] - a) % nk3[0]) * nk3[1] + (nk3[1] - b) % nk3[1]) * nk3[2] + (nk3[2] - c) % nk3[2];
  }
  SOX_CUDA_TRY(cudaMemcpyAsync(negm, h_neg.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, s));
  SOX_CUDA_TRY(cudaMemsetAsync(info, 0, 4 * sizeof(int), s));
  SOX_CUDA_TRY(cudaMemsetAsync(H, 0, sizeof(z) * (size_t)nk * nO * NN, s));
  // Frequencies in +-pairs (row nO-1-o of T_fwd the conjugate of row o) and G Hermitian give
  // Pi^q(-Omega) = Pi^q(Omega)^H and W_d^q(-Omega) = W_d^q(Omega)^H: only o < ns are solved.
  // A real molecule's bubble (the real part, symmetrised) needs the frequency pairs only.
  int ns = nO;
  {
    std::vector<double> hT(2 * (size_t)nO * T);
    unsigned long long hh[2] = {0, 0};
    SOX_CUDA_TRY(cudaMemcpyAsync(hT.data(), Tfd, sizeof(double) * hT.size(), cudaMemcpyDeviceToHost, s));
    if (!real) {
      SOX_CUDA_TRY(cudaMemsetAsync(hdev, 0, 2 * sizeof(unsigned long long), s));
      k_herm_dev<<<grid_of((long long)S * nk * T * nn), 256, 0, s>>>(G, n, (long long)S * nk * T, hdev);
      SOX_CUDA_TRY(cudaMemcpyAsync(hh, hdev, sizeof(hh), cudaMemcpyDeviceToHost, s));
    }
    SOX_CUDA_TRY(cudaStreamSynchronize(s));
    double tmax = 0.0, tdev = 0.0;
    for (int o = 0; o < nO; ++o)
      for (int j = 0; j < T; ++j) {
        const double *a = &hT[2 * ((size_t)o * T + j)], *b = &hT[2 * ((size_t)(nO - 1 - o) * T + j)];
        tmax = std::max(tmax, std::max(std::fabs(a[0]), std::fabs(a[1])));
        tdev = std::max(tdev, std::max(std::fabs(a[0] - b[0]), std::fabs(a[1] + b[1])));
      }
    double gmax = 0.0, gdev = 0.0;
    std::memcpy(&gmax, &hh[0], sizeof(double));
    std::memcpy(&gdev, &hh[1], sizeof(double));
    const bool pairs = tdev <= 1e-12 * tmax;
    const bool herm = real || gdev <= 1e-12 * gmax;
    if (pairs && herm) ns = (nO + 1) / 2;
  }
  ProfScope ps(h, "w_dynamic", s, 0);
  long long launches = 0;
  const int n_chunks = (ns + kBubF - 1) / kBubF;   // the bubble of the frequencies solved
  for (int sp = 0; sp < S; ++sp) {
    for (int k = 0; k < nk; ++k) {
      ZGemm a = zg();   // GR[j] = X^k G^k(tau_j)
      a.M = N; a.Nc = n; a.K = n; a.batch = T;
      a.A = X + (long long)k * N * n; a.sA = 0; a.ai = n; a.ak = 1;
      a.B = G + ((long long)sp * nk + k) * T * nn; a.sB = nn; a.bk = n; a.bj = 1;
      a.C = GR; a.sC = (long long)N * n; a.ci = n; a.cj = 1;
      zgemm(a, s);
      ZGemm b = zg();   // A_k(tau_j) = GR[j] X^k^H
      b.M = N; b.Nc = N; b.K = n; b.batch = T;
      b.A = GR; b.sA = (long long)N * n; b.ai = n; b.ak = 1;
      b.B = X + (long long)k * N * n; b.sB = 0; b.bk = 1; b.bj = n; b.conjB = 1;
      b.C = Ah + (long long)k * T * NN; b.sC = NN; b.ci = N; b.cj = 1;
      zgemm(b, s);
      launches += 2;
    }
    mesh_dft(Ah, (long long)T * NN, (long long)T * NN, nk3, -1, s);   // A-hat(m) = sum_k w^{-m.k} A_k
    dim3 grid((N + 31) / 32, (N + 31) / 32, (unsigned)(nk * n_chunks));
    k_bubble_reduce<<<grid, 256, 0, s>>>(Ah, Tf, negm, N, T, nO, ns, n_chunks, -1.0 / ((double)nk * nk), H);
    launches += 4;
  }
  mesh_dft(H, (long long)ns * NN, (long long)nO * NN, nk3, 1, s);   // Pi^q = sum_m w^{+m.q} H(m), o < ns
  if (real) k_sym_real<<<grid_of((long long)ns * NN), 256, 0, s>>>(H, N, ns);
  const int batch = nk * ns;
  k_gj_init_c<<<grid_of((long long)batch * NN), 256, 0, s>>>(V, N, ns, batch, Aug);
  for (int q = 0; q < nk; ++q) {   // left half: I - V^q Pi^q(i Omega_o), o < ns
    ZGemm g = zg();
    g.M = N; g.Nc = N; g.K = N; g.batch = ns;
    g.A = V + (long long)q * NN; g.sA = 0; g.ai = N; g.ak = 1;
    g.B = H + (long long)q * nO * NN; g.sB = NN; g.bk = N; g.bj = 1;
    g.C = Aug + (long long)q * ns * 2 * NN; g.sC = 2 * NN; g.ci = 2LL * N; g.cj = 1;
    g.alpha = -1.0; g.beta = 1.0;
    zgemm(g, s);
  }
  for (int k = 0; k < N; ++k) {
    k_gj_pivot_c<<<batch, 256, 0, s>>>(Aug, N, k, info);
    const int ncols = 2 * N - (k + 1);
    k_gj_elim_c<<<dim3((ncols + 255) / 256, std::min(N, 64), batch), 256, 0, s>>>(Aug, N, k, info);
  }
  k_gj_out<<<grid_of((long long)batch * NN), 256, 0, s>>>(Aug, V, N, nO, ns, batch, real ? 1 : 0, Wd);
  if (ns < nO)
    k_w_mirror<<<grid_of((long long)nk * (nO - ns) * NN), 256, 0, s>>>(Wd, N, nO, ns, nk, real ? 1 : 0);
  h->launches += launches + 2LL * N + 4 + nk;
  SOX_CUDA_TRY(cudaGetLastError());
  int hinfo[4] = {0, 0, 0, 0};
  SOX_CUDA_TRY(cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, s));
  SOX_CUDA_TRY(cudaStreamSynchronize(s));
  if (hinfo[1]) return {SOX_ERR_INVALID_ARG, "1 - V Pi(i Omega) is singular"};
  return Status::ok();
}

}  // namespace sox
