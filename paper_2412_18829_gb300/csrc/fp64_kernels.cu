// FP64 CUDA-core kernels: the plain double-precision path of every step, and the
// FP64 steps of the mixed-precision path (projections, back-projection, traces,
// Pi(0), W(0)).
#include "internal.h"

namespace sox {
namespace {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

// Loads a TM x TK (rows x k) tile of a strided operand into s[TK][TM+1].
__device__ __forceinline__ void load_tile_rowsk(double (*s)[TM + 1], const double *base, long long rs,
                                                long long ks, int r0, int k0, int R, int K, int tid) {
  if (ks == 1) {
#pragma unroll
    for (int it = 0; it < (TM * TK) / NT; ++it) {
      int e = tid + it * NT;
      int r = e / TK, k = e % TK;
      int gr = r0 + r, gk = k0 + k;
      s[k][r] = (gr < R && gk < K) ? base[gr * rs + gk] : 0.0;
    }
  } else {
#pragma unroll
    for (int it = 0; it < (TM * TK) / NT; ++it) {
      int e = tid + it * NT;
      int r = e % TM, k = e / TM;
      int gr = r0 + r, gk = k0 + k;
      s[k][r] = (gr < R && gk < K) ? base[gr * rs + gk * ks] : 0.0;
    }
  }
}

__global__ void __launch_bounds__(NT) k_gemm_f64(GemmF64 g) {
  __shared__ double sa[TK][TM + 1];
  __shared__ double sb[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
  const long long b = blockIdx.z;
  if (g.skip && g.skip[b]) return;
  const double *A = g.A + b * g.sA;
  const double *B = g.B + b * g.sB;
  double *C = g.C + b * g.sC;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < g.K; k0 += TK) {
    load_tile_rowsk(sa, A, g.ai, g.ak, i0, k0, g.M, g.K, tid);
    load_tile_rowsk(sb, B, g.bj, g.bk, j0, k0, g.Nc, g.K, tid);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sa[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = sb[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gi = i0 + ty + 16 * i;
    if (gi >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gj = j0 + tx + 16 * j;
      if (gj >= g.Nc) continue;
      double *c = C + gi * g.ci + gj * g.cj;
      double v = g.alpha * acc[i][j];
      if (g.beta != 0.0) v = fma(g.beta, *c, v);
      *c = v;
    }
  }
}

__global__ void k_pair_products(const double *X, double *Y, int N, int n) {
  long long total = (long long)N * n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int s = e % n;
    long long t = e / n;
    int q = t % n;
    int Q = t / n;
    Y[e] = X[(long long)Q * n + q] * X[(long long)Q * n + s];
  }
}

// Fused B/C/Hadamard-reduce over v for one (P,R) tile per CTA.
__global__ void __launch_bounds__(NT) k_sox_bcd_f64(const double *A, long long sA, const double *GR,
                                                   long long sGR, const double *GWt, long long sGW,
                                                   const double *U2, double *D, long long sD, int n,
                                                   int N, int v0, int v1) {
  __shared__ double s_a[TK][TM + 1];
  __shared__ double s_gr[TK][TN + 1];
  __shared__ double s_gw[TK][TM + 1];
  __shared__ double s_u[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int P0 = blockIdx.y * TM, R0 = blockIdx.x * TN;
  const long long b = blockIdx.z;
  const double *Ab = A + b * sA;
  const double *GRb = GR + b * sGR;
  const double *GWb = GWt + b * sGW;
  double d[4][4] = {};
  const long long nn = (long long)n * n;
  for (int v = v0; v < v1; ++v) {
    double bacc[4][4] = {}, cacc[4][4] = {};
    const double *Av = Ab + (long long)v * N * n;  // A[v][P][q]
    const double *Uv = U2 + (long long)v * n;      // U2[R][v][w], row stride n^2
    for (int k0 = 0; k0 < n; k0 += TK) {
      load_tile_rowsk(s_a, Av, n, 1, P0, k0, N, n, tid);
      load_tile_rowsk(s_gr, GRb, n, 1, R0, k0, N, n, tid);
      load_tile_rowsk(s_gw, GWb, n, 1, P0, k0, N, n, tid);
      load_tile_rowsk(s_u, Uv, nn, 1, R0, k0, N, n, tid);
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
        for (int j = 0; j < 4; ++j) {
          gr[j] = s_gr[kk][tx + 16 * j];
          u[j] = s_u[kk][tx + 16 * j];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            bacc[i][j] = fma(a[i], gr[j], bacc[i][j]);
            cacc[i][j] = fma(gw[i], u[j], cacc[i][j]);
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) d[i][j] = fma(bacc[i][j], cacc[i][j], d[i][j]);
  }
  double *Db = D + b * sD;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int P = P0 + ty + 16 * i;
    if (P >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int R = R0 + tx + 16 * j;
      if (R < N) Db[(long long)P * N + R] = d[i][j];
    }
  }
}

__device__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    int nw = (blockDim.x + 31) / 32;
    v = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// one block per (spin, tau)
__global__ void k_trace_sigma_gminus(const double *Sigma, const double *G, int n, int n_tau,
                                     double *partial) {
  const int j = blockIdx.x, s = blockIdx.y;
  const long long nn = (long long)n * n;
  const double *S = Sigma + ((long long)s * n_tau + j) * nn;
  const double *Gr = G + ((long long)s * n_tau + (n_tau - 1 - j)) * nn;
  double acc = 0.0;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    int t = e / n, r = e % n;
    acc = fma(S[e], -Gr[(long long)r * n + t], acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[(long long)s * n_tau + j] = acc;
}

__global__ void k_phi_finish(const double *partial, const double *w, int n_tau, int n_spin,
                             double *phi) {
  int s = threadIdx.x;
  if (s >= n_spin) return;
  double acc = 0.0;
  for (int j = 0; j < n_tau; ++j) acc = fma(w[j], partial[(long long)s * n_tau + j], acc);
  phi[s] = 0.25 * acc;
}

__global__ void k_dG_from_sigma(const double *Sigma, const double *w, const double *dphi, int n,
                                int n_tau, int n_spin, double *dG) {
  const long long nn = (long long)n * n;
  const long long total = nn * n_tau * n_spin;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long m = e / nn;
    int rt = e % nn;
    int r = rt / n, t = rt % n;
    int j = m % n_tau, s = m / n_tau;
    const double *S = Sigma + ((long long)s * n_tau + (n_tau - 1 - j)) * nn;
    dG[e] = -dphi[s] * w[j] * S[(long long)t * n + r];
  }
}

// 32 x 32 output tile per block, 256 threads (each 4 elements)
__global__ void k_pi0_reduce(const double *GPQ, const double *w, int N, int n_tau, double *Pi) {
  __shared__ double ta[32][33];
  __shared__ double tb[32][33];
  const int P0 = blockIdx.y * 32, Q0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // ty 0..7
  const long long NN = (long long)N * N;
  double acc[4] = {0, 0, 0, 0};
  for (int j = 0; j < n_tau; ++j) {
    const double *Aj = GPQ + j * NN;
    const double *Bj = GPQ + (long long)(n_tau - 1 - j) * NN;
    for (int r = ty; r < 32; r += 8) {
      int P = P0 + r, Q = Q0 + tx;
      ta[r][tx] = (P < N && Q < N) ? Aj[(long long)P * N + Q] : 0.0;
      int Qb = Q0 + r, Pb = P0 + tx;
      tb[r][tx] = (Qb < N && Pb < N) ? Bj[(long long)Qb * N + Pb] : 0.0;  // tb[Q][P]
    }
    __syncthreads();
    const double wj = w[j];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int r = ty + 8 * i;  // P offset
      acc[i] = fma(wj, ta[r][tx] * tb[tx][r], acc[i]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int P = P0 + ty + 8 * i, Q = Q0 + tx;
    if (P < N && Q < N) Pi[(long long)P * N + Q] = -acc[i];
  }
}

// Gauss-Jordan, step k, part 1 (one block): partial pivoting, row swap, scaling of row k.
__global__ void k_gj_pivot(double *Aug, int N, int k, int *info) {
  __shared__ double best[1024];
  __shared__ int bidx[1024];
  const long long W = 2LL * N;
  double bv = -1.0;
  int bi = k;
  for (int i = k + threadIdx.x; i < N; i += blockDim.x) {
    double a = fabs(Aug[i * W + k]);
    if (a > bv) { bv = a; bi = i; }
  }
  best[threadIdx.x] = bv;
  bidx[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double ov = best[threadIdx.x + o];
      int oi = bidx[threadIdx.x + o];
      if (ov > best[threadIdx.x] || (ov == best[threadIdx.x] && oi < bidx[threadIdx.x])) {
        best[threadIdx.x] = ov;
        bidx[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int p = bidx[0];
  const double pv = Aug[p * W + k];
  if (!(best[0] > 0.0)) {
    if (threadIdx.x == 0) info[1] = 1;
    return;
  }
  const double inv = 1.0 / pv;
  for (long long j = k + threadIdx.x; j < W; j += blockDim.x) {
    double a = Aug[(long long)k * W + j];
    double b = Aug[(long long)p * W + j];
    if (p != k) Aug[(long long)p * W + j] = a;
    Aug[(long long)k * W + j] = b * inv;
  }
}

// Gauss-Jordan, step k, part 2: eliminate column k from every other row
// (columns j > k of the left half and all of the right half).
__global__ void k_gj_elim(double *Aug, int N, int k, const int *info) {
  if (info[1]) return;
  const long long W = 2LL * N;
  const int ncols = (int)(W - (k + 1));
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  const long long col = k + 1 + j;
  const double rk = Aug[(long long)k * W + col];
  for (int i = blockIdx.y; i < N; i += gridDim.y) {
    if (i == k) continue;
    double f = Aug[(long long)i * W + k];
    Aug[(long long)i * W + col] = fma(-f, rk, Aug[(long long)i * W + col]);
  }
}

__global__ void k_build_gj(const double *V, double *Aug, int N) {
  const long long total = (long long)N * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = e / N, j = e % N;
    Aug[(long long)i * 2 * N + j] = (i == j) ? 1.0 : 0.0;
    Aug[(long long)i * 2 * N + N + j] = V[e];
  }
}

__global__ void k_copy_right(const double *Aug, double *W, int N) {
  const long long total = (long long)N * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = e / N, j = e % N;
    W[e] = Aug[(long long)i * 2 * N + N + j];
  }
}

__global__ void k_neg_reflect(const double *src, double *dst, long long mat, int n_tau, int count) {
  const long long total = mat * n_tau * count;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long m = e / mat, off = e % mat;
    int j = m % n_tau;
    long long c = m / n_tau;
    dst[e] = -src[(c * n_tau + (n_tau - 1 - j)) * mat + off];
  }
}

__global__ void k_symmetry_flags(const double *G, int n, int *flag) {
  const int b = blockIdx.x;
  const double *g = G + (long long)b * n * n;
  double m = 0.0, d = 0.0;
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    m = fmax(m, fabs(g[e]));
    d = fmax(d, fabs(g[e] - g[(long long)j * n + i]));
  }
  __shared__ double sm[256], sd[256];
  sm[threadIdx.x] = m;
  sd[threadIdx.x] = d;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
      sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) flag[b] = (sd[0] <= 1e-14 * sm[0]) ? 1 : 0;
}

__global__ void k_add(const double *a, const double *b, double *dst, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = a[e] + b[e];
}

inline int grid_for(long long total, int threads = 256) {
  long long b = (total + threads - 1) / threads;
  if (b > 65535LL * 16) b = 65535LL * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

void launch_gemm_f64(const GemmF64 &g, cudaStream_t s) {
  if (g.M <= 0 || g.Nc <= 0 || g.batch <= 0) return;
  dim3 grid((g.Nc + TN - 1) / TN, (g.M + TM - 1) / TM, g.batch);
  k_gemm_f64<<<grid, NT, 0, s>>>(g);
}

void launch_pair_products_f64(const double *X, double *Y, int N, int n, cudaStream_t s) {
  long long total = (long long)N * n * n;
  k_pair_products<<<grid_for(total), 256, 0, s>>>(X, Y, N, n);
}

void launch_sox_bcd_f64(const double *A, long long sA, const double *GR, long long sGR,
                        const double *GWt, long long sGW, const double *U2, double *D,
                        long long sD, int n, int N, int batch, cudaStream_t s, int v0, int v1) {
  dim3 grid((N + TN - 1) / TN, (N + TM - 1) / TM, batch);
  v1 = (v1 <= 0 || v1 > n) ? n : v1;
  v0 = v0 < 0 ? 0 : (v0 > v1 ? v1 : v0);
  k_sox_bcd_f64<<<grid, NT, 0, s>>>(A, sA, GR, sGR, GWt, sGW, U2, D, sD, n, N, v0, v1);
}

void launch_trace_sigma_gminus(const double *Sigma, const double *G, int n, int n_tau,
                               int n_spin, double *partial, cudaStream_t s) {
  k_trace_sigma_gminus<<<dim3(n_tau, n_spin), 256, 0, s>>>(Sigma, G, n, n_tau, partial);
}

void launch_phi_finish(const double *partial, const double *w, int n_tau, int n_spin,
                       double *phi, cudaStream_t s) {
  k_phi_finish<<<1, 32, 0, s>>>(partial, w, n_tau, n_spin, phi);
}

void launch_dG_from_sigma(const double *Sigma, const double *w, const double *dphi, int n,
                          int n_tau, int n_spin, double *dG, cudaStream_t s) {
  long long total = (long long)n * n * n_tau * n_spin;
  k_dG_from_sigma<<<grid_for(total), 256, 0, s>>>(Sigma, w, dphi, n, n_tau, n_spin, dG);
}

void launch_pi0_reduce(const double *GPQ, const double *w, int N, int n_tau, double *Pi,
                       cudaStream_t s) {
  dim3 grid((N + 31) / 32, (N + 31) / 32);
  k_pi0_reduce<<<grid, 256, 0, s>>>(GPQ, w, N, n_tau, Pi);
}

void launch_gj_step(double *Aug, int N, int k, int *info, cudaStream_t s) {
  k_gj_pivot<<<1, 1024, 0, s>>>(Aug, N, k, info);
  int ncols = 2 * N - (k + 1);
  dim3 grid((ncols + 255) / 256, N < 256 ? N : 256);
  k_gj_elim<<<grid, 256, 0, s>>>(Aug, N, k, info);
}

void launch_build_gj_system(const double *V, const double *Pi, double *Aug, int N, cudaStream_t s) {
  k_build_gj<<<grid_for((long long)N * N), 256, 0, s>>>(V, Aug, N);
  // left half: I - V Pi
  GemmF64 g;
  g.M = N; g.Nc = N; g.K = N;
  g.A = V; g.ai = N; g.ak = 1;
  g.B = Pi; g.bk = N; g.bj = 1;
  g.C = Aug; g.ci = 2LL * N; g.cj = 1;
  g.alpha = -1.0; g.beta = 1.0;
  launch_gemm_f64(g, s);
}

void launch_copy_right_half(const double *Aug, double *W, int N, cudaStream_t s) {
  k_copy_right<<<grid_for((long long)N * N), 256, 0, s>>>(Aug, W, N);
}

void launch_add_f64(const double *a, const double *b, double *dst, long long count, cudaStream_t s) {
  k_add<<<grid_for(count), 256, 0, s>>>(a, b, dst, count);
}

void launch_symmetry_flags(const double *G, int n, int batch, int *flag, cudaStream_t s) {
  k_symmetry_flags<<<batch, 256, 0, s>>>(G, n, flag);
}

void launch_neg_reflect(const double *src, double *dst, long long mat, int n_tau, int count,
                        cudaStream_t s) {
  k_neg_reflect<<<grid_for(mat * n_tau * count), 256, 0, s>>>(src, dst, mat, n_tau, count);
}

}  // namespace sox
