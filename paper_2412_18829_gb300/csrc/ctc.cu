// Complex split-precision GEMMs on the tensor cores, and the momentum-resolved
// SOX chain of Sec. II C (static, and the dynamic algorithm with momenta) on them.
//
// A complex product C[i][j] = sum_k A[i][k] B[j][k] runs as ONE real GEMM of the
// FP16-pair kernel: a row of A is its interleaved (re, im) values (2K reals); each
// complex row j of B becomes two real rows,
//   re-row (b_r, -sa sb b_i) and im-row (sb b_i, sa b_r)   (sa, sb = -1 for conj(A), conj(B)),
// so the real output row holds (Re C[i][j], Im C[i][j]) interleaved: the library's
// complex layout.  Every split row carries a power-of-two scale; the GEMM epilogue
// multiplies the FP32 accumulators back by the row and column factors.
#include <algorithm>
#include <vector>

#include "ctc.h"
#include "kpoint.h"
#include "tc_common.cuh"
#include "tc_kernels.h"

namespace sox {
namespace {

__device__ __forceinline__ float cwarp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double2 ld_c(const double2 *p) { return *p; }
__device__ __forceinline__ double2 ld_c(const float2 *p) {
  const float2 v = *p;
  return make_double2(v.x, v.y);
}

// FP16 pair of x * s (s a power of two, exact in FP64): hi rounds to nearest.
__device__ __forceinline__ void split_pair(double x, float s, __half &h, __half &l) {
  const double xs = x * (double)s;
  h = __float2half_rn((float)xs);
  l = __float2half_rn((float)(xs - (double)__half2float(h)));
}

// Row r of batch b starts at src + b*sb + (r / R2)*sr1 + (r % R2)*sr2; its k-th complex
// element is k*sk further (all in complex elements).
struct RowMap {
  long long sb, sr1, sr2, sk;
  int R2;
  __device__ __forceinline__ long long row(int b, int r) const {
    return (long long)b * sb + (long long)(r / R2) * sr1 + (long long)(r % R2) * sr2;
  }
};

// A operand: one warp per complex row -> one real row of 2K interleaved values.
template <class T>
__global__ void k_csplit_a(const T *src, RowMap m, int batch, int rows, int K, int Kp2, __half *hi, __half *lo,
                           float *unscale) {
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (gw >= (long long)rows * batch) return;
  const int b = (int)(gw / rows), r = (int)(gw % rows);
  const T *x = src + m.row(b, r);
  float mx = 0.f;
  for (int k = lane; k < K; k += 32) {
    const double2 v = ld_c(x + k * m.sk);
    mx = fmaxf(mx, fmaxf((float)fabs(v.x), (float)fabs(v.y)));
  }
  mx = cwarp_max(mx);
  const float s = tc::pow2_floor_inv(mx);
  __half *h = hi + gw * Kp2, *l = lo + gw * Kp2;
  for (int c = lane; c < Kp2; c += 32) {
    __half a = __float2half(0.f), d = __float2half(0.f);
    const int k = c >> 1;
    if (k < K) {
      const double2 v = ld_c(x + k * m.sk);
      split_pair((c & 1) ? v.y : v.x, s, a, d);
    }
    h[c] = a;
    l[c] = d;
  }
  if (lane == 0) unscale[gw] = 1.f / s;
}

// B operand: one warp per complex row j -> real rows 2j (re-row) and 2j+1 (im-row).
template <class T>
__global__ void k_csplit_b(const T *src, RowMap m, int batch, int cols, int K, int Kp2, float sa, float sbc,
                           __half *hi, __half *lo, float *unscale) {
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (gw >= (long long)cols * batch) return;
  const int b = (int)(gw / cols), j = (int)(gw % cols);
  const T *x = src + m.row(b, j);
  float mx = 0.f;
  for (int k = lane; k < K; k += 32) {
    const double2 v = ld_c(x + k * m.sk);
    mx = fmaxf(mx, fmaxf((float)fabs(v.x), (float)fabs(v.y)));
  }
  mx = cwarp_max(mx);
  const float s = tc::pow2_floor_inv(mx);
  const long long r0 = ((long long)b * cols + j) * 2;
  __half *h0 = hi + r0 * Kp2, *l0 = lo + r0 * Kp2;
  __half *h1 = h0 + Kp2, *l1 = l0 + Kp2;
  for (int c = lane; c < Kp2; c += 32) {
    __half a0 = __float2half(0.f), d0 = __float2half(0.f), a1 = __float2half(0.f), d1 = __float2half(0.f);
    const int k = c >> 1;
    if (k < K) {
      const double2 v = ld_c(x + k * m.sk);
      const double re = (c & 1) ? -(double)(sa * sbc) * v.y : v.x;
      const double im = (c & 1) ? (double)sa * v.x : (double)sbc * v.y;
      split_pair(re, s, a0, d0);
      split_pair(im, s, a1, d1);
    }
    h0[c] = a0;
    l0[c] = d0;
    h1[c] = a1;
    l1[c] = d1;
  }
  if (lane == 0) unscale[r0] = unscale[r0 + 1] = 1.f / s;
}

// The n_k^3 D step on FP32 complex B and C, one tile of E consecutive (P, R) elements
// per block with all n_k^2 pairs of both in shared memory:
//   D[i][k][e] += sum_{q1,q2} C[i][(q2, k+q1)][e] * B[i][(q1, k+q1-q2)][e]
// (FP32 sum over the n_k^2 products of one v, added to the FP64 D).
// B, C: float2, element e of pair p and chunk index il at p * sP + il * sI + e; D: double2
// [i][k][NN] at D + (i0 + il) * sDi.
__global__ void k_kpoint_D_blk(const float2 *B, const float2 *C, long long sP, long long sI, const int *add,
                               const int *sub, int nk, long long NN, int E, int i0, long long sDi, double2 *D) {
  extern __shared__ float2 sm[];
  const int np = nk * nk;
  float2 *sB = sm, *sC = sm + (size_t)np * E;
  const int il = blockIdx.y;
  const long long e0 = (long long)blockIdx.x * E;
  const int ne = (int)std::min<long long>(E, NN - e0);
  const float2 *Bi = B + (long long)il * sI, *Ci = C + (long long)il * sI;
  for (int t = threadIdx.x; t < np * E; t += blockDim.x) {
    const int pr = t / E, e = t % E;
    float2 zb = make_float2(0.f, 0.f), zc = zb;
    if (e < ne) {
      zb = Bi[(long long)pr * sP + e0 + e];
      zc = Ci[(long long)pr * sP + e0 + e];
    }
    sB[t] = zb;
    sC[t] = zc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nk * E; t += blockDim.x) {
    const int k = t / E, e = t % E;
    if (e >= ne) continue;
    float ar = 0.f, ai = 0.f;
    for (int q1 = 0; q1 < nk; ++q1) {
      const int kw = add[k * nk + q1];
      for (int q2 = 0; q2 < nk; ++q2) {
        const int ks = sub[kw * nk + q2];
        const float2 c = sC[(q2 * nk + kw) * E + e];
        const float2 b = sB[(q1 * nk + ks) * E + e];
        ar = fmaf(c.x, b.x, fmaf(-c.y, b.y, ar));
        ai = fmaf(c.x, b.y, fmaf(c.y, b.x, ai));
      }
    }
    double2 *d = D + (long long)(i0 + il) * sDi + (long long)k * NN + e0 + e;
    double2 v = *d;
    v.x += ar;
    v.y += ai;
    *d = v;
  }
}

// B operand of the mixed tensor, built from X directly: for pair (q, k') and row (a, b),
//   y[Q] = conj(X^{k'-q}[Q][a]) X^{k'}[Q][b],  re-row (y_r, -y_i), im-row (y_i, y_r), K = Q.
__global__ void k_csplit_pairs(const double2 *X, const int *sub, int nk, int N, int n, int Kp2, __half *hi,
                               __half *lo, float *unscale) {
  const long long nn = (long long)n * n;
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (gw >= nn * nk * nk) return;
  const int pr = (int)(gw / nn), ab = (int)(gw % nn);
  const int a = ab / n, bb = ab % n;
  const int q = pr / nk, kk = pr % nk;
  const double2 *Xa = X + (long long)sub[kk * nk + q] * N * n + a;
  const double2 *Xb = X + (long long)kk * N * n + bb;
  auto y = [&](int Q) {
    const double2 u = Xa[(long long)Q * n], w = Xb[(long long)Q * n];
    return make_double2(u.x * w.x + u.y * w.y, u.x * w.y - u.y * w.x);
  };
  float mx = 0.f;
  for (int Q = lane; Q < N; Q += 32) {
    const double2 v = y(Q);
    mx = fmaxf(mx, fmaxf((float)fabs(v.x), (float)fabs(v.y)));
  }
  mx = cwarp_max(mx);
  const float s = tc::pow2_floor_inv(mx);
  const long long r0 = gw * 2;
  __half *h0 = hi + r0 * Kp2, *l0 = lo + r0 * Kp2;
  __half *h1 = h0 + Kp2, *l1 = l0 + Kp2;
  for (int c = lane; c < Kp2; c += 32) {
    __half a0 = __float2half(0.f), d0 = a0, a1 = a0, d1 = a0;
    const int Q = c >> 1;
    if (Q < N) {
      const double2 v = y(Q);
      split_pair((c & 1) ? -v.y : v.x, s, a0, d0);
      split_pair((c & 1) ? v.x : v.y, s, a1, d1);
    }
    h0[c] = a0;
    l0[c] = d0;
    h1[c] = a1;
    l1[c] = d1;
  }
  if (lane == 0) unscale[r0] = unscale[r0 + 1] = 1.f / s;
}

int blocks_for(long long warps) { return (int)std::max<long long>(1, (warps * 32 + 255) / 256); }

}  // namespace

int csplit_kp2(int K) { return ((2 * K + 63) / 64) * 64; }

size_t csplit_bytes(int batch, int rows_real, int K) {
  const size_t e = (size_t)batch * rows_real * csplit_kp2(K);
  return 2 * aligned_bytes(e, 2) + aligned_bytes((size_t)batch * rows_real, 4);
}

CSplit csplit_take(Arena &ar, int batch, int rows_real, int K) {
  CSplit c;
  c.batch = batch;
  c.rows = rows_real;
  c.Kp2 = csplit_kp2(K);
  const size_t e = (size_t)batch * rows_real * c.Kp2;
  c.hi = ar.take<__half>(e);
  c.lo = ar.take<__half>(e);
  c.unscale = ar.take<float>((size_t)batch * rows_real);
  if (!c.unscale) c.hi = nullptr;
  return c;
}

void csplit_a(const void *src, bool f32, long long sb, long long sr1, long long sr2, int R2, long long sk, int batch,
              int rows, int K, const CSplit &out, cudaStream_t s) {
  RowMap m{sb, sr1, sr2, sk, R2 > 0 ? R2 : 1};
  if (R2 <= 0) {
    m.sr1 = sr1;
    m.sr2 = 0;
    m.R2 = 1;
  }
  const int blocks = blocks_for((long long)rows * batch);
  if (f32)
    k_csplit_a<float2><<<blocks, 256, 0, s>>>(static_cast<const float2 *>(src), m, batch, rows, K, out.Kp2, out.hi,
                                              out.lo, out.unscale);
  else
    k_csplit_a<double2><<<blocks, 256, 0, s>>>(static_cast<const double2 *>(src), m, batch, rows, K, out.Kp2, out.hi,
                                               out.lo, out.unscale);
}

void csplit_b(const void *src, bool f32, long long sb, long long sr1, long long sr2, int R2, long long sk, int batch,
              int cols, int K, bool conjA, bool conjB, const CSplit &out, cudaStream_t s) {
  RowMap m{sb, sr1, sr2, sk, R2 > 0 ? R2 : 1};
  if (R2 <= 0) {
    m.sr1 = sr1;
    m.sr2 = 0;
    m.R2 = 1;
  }
  const int blocks = blocks_for((long long)cols * batch);
  const float sa = conjA ? -1.f : 1.f, sbc = conjB ? -1.f : 1.f;
  if (f32)
    k_csplit_b<float2><<<blocks, 256, 0, s>>>(static_cast<const float2 *>(src), m, batch, cols, K, out.Kp2, sa, sbc,
                                              out.hi, out.lo, out.unscale);
  else
    k_csplit_b<double2><<<blocks, 256, 0, s>>>(static_cast<const double2 *>(src), m, batch, cols, K, out.Kp2, sa,
                                               sbc, out.hi, out.lo, out.unscale);
}

void csplit_pairs(const double *X, const int *sub, int nk, int N, int n, const CSplit &out, cudaStream_t s) {
  const long long warps = (long long)n * n * nk * nk;
  k_csplit_pairs<<<blocks_for(warps), 256, 0, s>>>(reinterpret_cast<const double2 *>(X), sub, nk, N, n, out.Kp2, out.hi,
                                                   out.lo, out.unscale);
}

Status cgemm_tc(sox_handle h, const CSplit &A, const CSplit &B, int batch, const int *idxA, const int *idxB,
                float alpha, float *C, long long ldc, long long sCb, cudaStream_t s) {
  if (batch <= 0 || A.rows <= 0 || B.rows <= 0) return Status::ok();
  if (A.Kp2 != B.Kp2) return {SOX_ERR_INVALID_ARG, "cgemm_tc: operands split with different K"};
  if ((ldc & 3) || (sCb & 3) || (reinterpret_cast<uintptr_t>(C) & 15))
    return {SOX_ERR_INVALID_ARG, "cgemm_tc: output not 16-byte aligned"};
  CUtensorMap maps[6];
  std::string err;
  const long long bsA = A.bstride ? A.bstride : A.rows, bsB = B.bstride ? B.bstride : B.rows;
  if (!make_tmap_f16_3d_bs(&maps[0], A.hi, A.Kp2, A.rows, A.batch, bsA * A.Kp2, 64, 128, &err) ||
      !make_tmap_f16_3d_bs(&maps[1], A.lo, A.Kp2, A.rows, A.batch, bsA * A.Kp2, 64, 128, &err) ||
      !make_tmap_f16_3d_bs(&maps[2], B.hi, B.Kp2, B.rows, B.batch, bsB * B.Kp2, 64, 128, &err) ||
      !make_tmap_f16_3d_bs(&maps[3], B.lo, B.Kp2, B.rows, B.batch, bsB * B.Kp2, 64, 128, &err))
    return {SOX_ERR_CUDA, "cgemm_tc: " + err};
  maps[4] = maps[0];   // no TMA stores in FP32 mode; valid maps for the prefetch
  maps[5] = maps[1];
  GemmTcArgs ga;
  ga.M = A.rows;
  ga.Ncols = B.rows;
  ga.Kp = A.Kp2;
  ga.batch = batch;
  ga.batchA_shared = (A.batch == 1);
  ga.batchB_shared = (B.batch == 1);
  ga.idxA = idxA;
  ga.idxB = idxB;
  ga.mode = kStoreF32;
  ga.Cf = C;
  ga.ldc = ldc;
  ga.sCb = sCb;
  ga.alpha = alpha;
  ga.row_scale = A.unscale;
  ga.rs_b = bsA;
  ga.col_scale = B.unscale;
  ga.cs_b = bsB;
  ga.spin_limit = h->spin_limit;
  ga.status = h->d_status;
  const long long tiles = (long long)batch * ((A.rows + 127) / 128) * ((B.rows + 127) / 128);
  const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, h->sm_count));
  ++h->launches;
  SOX_CUDA_TRY(launch_gemm_f16x2(maps, ga, grid, s));
  return Status::ok();
}

Status kpoint_D_f32(const float *B, const float *C, long long sP, long long sI, const int *add, const int *sub,
                    int nk, long long NN, int ct, int i0, long long sDi, double *D, cudaStream_t s) {
  const long long np = (long long)nk * nk;
  const size_t per_e = (size_t)np * 2 * sizeof(float2);
  const size_t cap = 96 * 1024;
  if (per_e > cap) return {SOX_ERR_SHAPE, "k-mesh too large for the split-precision D step"};
  const int E = (int)std::min<size_t>(8, cap / per_e);
  static bool attr = false;
  if (!attr) {
    SOX_CUDA_TRY(cudaFuncSetAttribute(k_kpoint_D_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
    attr = true;
  }
  dim3 grid((unsigned)((NN + E - 1) / E), (unsigned)ct);
  k_kpoint_D_blk<<<grid, 256, per_e * E, s>>>(reinterpret_cast<const float2 *>(B), reinterpret_cast<const float2 *>(C),
                                              sP, sI, add, sub, nk, NN, E, i0, sDi, reinterpret_cast<double2 *>(D));
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

}  // namespace sox
