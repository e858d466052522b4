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

// loads keep the source precision: FP32 sources are split in FP32 arithmetic (exact: the
// scale is a power of two and hi's remainder is representable), FP64 sources in FP64
__device__ __forceinline__ double2 ld_c(const double2 *p) { return *p; }
__device__ __forceinline__ float2 ld_c(const float2 *p) { return *p; }

// FP16 pair of x * s (s a power of two): hi rounds to nearest, lo holds the remainder.
__device__ __forceinline__ void split_pair(float x, float s, __half &h, __half &l) {
  const float xs = x * s;
  h = __float2half_rn(xs);
  l = __float2half_rn(xs - __half2float(h));
}
__device__ __forceinline__ void split_pair(double x, float s, __half &h, __half &l) {
  const double xs = x * (double)s;
  h = __float2half_rn((float)xs);
  l = __float2half_rn((float)(xs - (double)__half2float(h)));
}
// rounding to nearest is symmetric, so the pair of -x is the negated pair of x: a B row's
// four signed copies of (b_r, b_i) take two splits
__device__ __forceinline__ __half neg_if(bool n, __half v) { return n ? __hneg(v) : v; }

__device__ __forceinline__ uint32_t pack_h2(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// Eight FP16 pairs (4 complex values, interleaved) of an A row -> one 16-byte store each
// for hi and lo.  v[j] are the complex values k0..k0+3 (zero beyond K).
template <class V2>
__device__ __forceinline__ void store8_a(const V2 *v, float s, __half *h, __half *l) {
  uint32_t ph[4], pl[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    __half a0, d0, a1, d1;
    split_pair(v[j].x, s, a0, d0);
    split_pair(v[j].y, s, a1, d1);
    ph[j] = pack_h2(a0, a1);
    pl[j] = pack_h2(d0, d1);
  }
  *reinterpret_cast<uint4 *>(h) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
  *reinterpret_cast<uint4 *>(l) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
}

// The same for the re-row and im-row of a B row: re (b_r, -sa sb b_i), im (sb b_i, sa b_r).
template <class V2>
__device__ __forceinline__ void store8_b(const V2 *v, float s, float sa, float sbc, __half *h0, __half *l0,
                                         __half *h1, __half *l1) {
  uint32_t p0[4], q0[4], p1[4], q1[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    __half xh, xl, yh, yl;
    split_pair(v[j].x, s, xh, xl);
    split_pair(v[j].y, s, yh, yl);
    const bool n_re = sa * sbc > 0.f, n_im = sbc < 0.f, n_x = sa < 0.f;
    p0[j] = pack_h2(xh, neg_if(n_re, yh));   // (b_r, -sa sb b_i)
    q0[j] = pack_h2(xl, neg_if(n_re, yl));
    p1[j] = pack_h2(neg_if(n_im, yh), neg_if(n_x, xh));   // (sb b_i, sa b_r)
    q1[j] = pack_h2(neg_if(n_im, yl), neg_if(n_x, xl));
  }
  *reinterpret_cast<uint4 *>(h0) = make_uint4(p0[0], p0[1], p0[2], p0[3]);
  *reinterpret_cast<uint4 *>(l0) = make_uint4(q0[0], q0[1], q0[2], q0[3]);
  *reinterpret_cast<uint4 *>(h1) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
  *reinterpret_cast<uint4 *>(l1) = make_uint4(q1[0], q1[1], q1[2], q1[3]);
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

// Lanes per row (a power of two dividing 32): a row of Kp2 halves is Kp2/8 16-byte
// chunks; short rows share a warp.
__host__ __device__ __forceinline__ int lanes_per_row(int Kp2) { return Kp2 >= 256 ? 32 : (Kp2 >= 128 ? 16 : 8); }

__device__ __forceinline__ float group_max(float v, int lpr) {
  for (int o = lpr / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// A operand: LPR lanes per complex row -> one real row of 2K interleaved values.
template <class T>
__global__ void k_csplit_a(const T *src, RowMap m, int batch, int rows, int K, int Kp2, __half *hi, __half *lo,
                           float *unscale) {
  const int lpr = lanes_per_row(Kp2);
  const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gr = gt / lpr;                 // row of this lane group
  const int gl = (int)(gt % lpr);
  const bool live = gr < (long long)rows * batch;
  const int b = live ? (int)(gr / rows) : 0, r = live ? (int)(gr % rows) : 0;
  const T *x = src + m.row(b, r);
  float mx = 0.f;
  if (live)
    for (int k = gl; k < K; k += lpr) {
      const T v = ld_c(x + k * m.sk);
      mx = fmaxf(mx, fmaxf((float)fabs(v.x), (float)fabs(v.y)));
    }
  mx = group_max(mx, lpr);
  if (!live) return;
  const float s = tc::pow2_floor_inv(mx);
  __half *h = hi + gr * Kp2, *l = lo + gr * Kp2;
  for (int c8 = gl; c8 < Kp2 / 8; c8 += lpr) {
    T v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = c8 * 4 + j;
      v[j] = k < K ? ld_c(x + k * m.sk) : T{};
    }
    store8_a(v, s, h + c8 * 8, l + c8 * 8);
  }
  if (gl == 0) unscale[gr] = 1.f / s;
}

// B operand: LPR lanes per complex row j -> real rows 2j (re-row) and 2j+1 (im-row).
template <class T>
__global__ void k_csplit_b(const T *src, RowMap m, int batch, int cols, int K, int Kp2, float sa, float sbc,
                           __half *hi, __half *lo, float *unscale) {
  const int lpr = lanes_per_row(Kp2);
  const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gr = gt / lpr;
  const int gl = (int)(gt % lpr);
  const bool live = gr < (long long)cols * batch;
  const int b = live ? (int)(gr / cols) : 0, j = live ? (int)(gr % cols) : 0;
  const T *x = src + m.row(b, j);
  float mx = 0.f;
  if (live)
    for (int k = gl; k < K; k += lpr) {
      const T v = ld_c(x + k * m.sk);
      mx = fmaxf(mx, fmaxf((float)fabs(v.x), (float)fabs(v.y)));
    }
  mx = group_max(mx, lpr);
  if (!live) return;
  const float s = tc::pow2_floor_inv(mx);
  const long long r0 = gr * 2;
  __half *h0 = hi + r0 * Kp2, *l0 = lo + r0 * Kp2;
  __half *h1 = h0 + Kp2, *l1 = l0 + Kp2;
  for (int c8 = gl; c8 < Kp2 / 8; c8 += lpr) {
    T v[4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int k = c8 * 4 + jj;
      v[jj] = k < K ? ld_c(x + k * m.sk) : T{};
    }
    store8_b(v, s, sa, sbc, h0 + c8 * 8, l0 + c8 * 8, h1 + c8 * 8, l1 + c8 * 8);
  }
  if (gl == 0) unscale[r0] = unscale[r0 + 1] = 1.f / s;
}

// The n_k^3 D step for any mesh (the fallback of the register forms below), one tile of E
// consecutive (P, R) elements per block with all n_k^2 pairs of both in shared memory:
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
  for (int c8 = lane; c8 < Kp2 / 8; c8 += 32) {
    double2 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int Q = c8 * 4 + j;
      v[j] = Q < N ? y(Q) : make_double2(0.0, 0.0);
    }
    store8_b(v, s, 1.f, 1.f, h0 + c8 * 8, l0 + c8 * 8, h1 + c8 * 8, l1 + c8 * 8);
  }
  if (lane == 0) unscale[r0] = unscale[r0 + 1] = 1.f / s;
}

// The D step with one thread per (P, R) element and all NK accumulators in registers:
// for every (k_s, k_w), c = C[(k_w - k_s, k_w)][e] is loaded once and multiplied with
// B[(k_w - k, k_s)][e] for every k.  Tables in shared memory; B and C read straight from
// global memory (coalesced along e), each B value reused from L1 NK times.
template <int NK>
__global__ void __launch_bounds__(128) k_kpoint_D_reg(const float2 *B, const float2 *C, long long sP, long long sI,
                                                     const int *add, const int *sub, long long NN, int i0,
                                                     long long sDi, double2 *D) {
  __shared__ int s_sub[NK * NK];
  for (int t = threadIdx.x; t < NK * NK; t += blockDim.x) s_sub[t] = sub[t];
  __syncthreads();
  const int il = blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NN) return;
  const float2 *Bi = B + (long long)il * sI + e, *Ci = C + (long long)il * sI + e;
  float ar[NK], ai[NK];
#pragma unroll
  for (int k = 0; k < NK; ++k) ar[k] = ai[k] = 0.f;
  // k_s outermost: the NK values B[(., k_s)][e] stay in L1 while k_w and k sweep them
  for (int ks = 0; ks < NK; ++ks) {
    for (int kw = 0; kw < NK; ++kw) {
      const int q2 = s_sub[kw * NK + ks];
      const float2 c = __ldg(Ci + (long long)(q2 * NK + kw) * sP);
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        const int q1 = s_sub[kw * NK + k];
        const float2 b = __ldg(Bi + (long long)(q1 * NK + ks) * sP);
        ar[k] = fmaf(c.x, b.x, fmaf(-c.y, b.y, ar[k]));
        ai[k] = fmaf(c.x, b.y, fmaf(c.y, b.x, ai[k]));
      }
    }
  }
  (void)add;
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    double2 *d = D + (long long)(i0 + il) * sDi + (long long)k * NN + e;
    double2 v = *d;
    v.x += ar[k];
    v.y += ai[k];
    *d = v;
  }
}

// The D step through the convolution theorem on the k mesh.  For one (P, R) element and
// one k_s, with c(x) = C[(x - k_s, x)] and b(y) = B[(y, k_s)],
//   D[k] += sum_x c(x) b(x - k),
// a cyclic cross-correlation over Z_N1 x Z_N2 x Z_N3.  With F-(m) = sum_x f(x) w^{-m.x},
// F+(m) = sum_x f(x) w^{+m.x}:  Dhat(m) = sum_{k_s} c^-(m) b^+(m), and
// D[k] = (1/n_k) sum_m w^{+m.k} Dhat(m): n_k^2 products per element instead of n_k^3, and
// for mesh sides up to 4 the small DFTs need additions only (sides of 3: one real scale).
// Thread (e, m1) owns one slab m1 of Dhat: the side-N1 transform is folded into the loads,
// the N2 x N3 transform runs in registers; the inverse side-N1 transform at the end goes
// through shared memory.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// v * i^sgn
__device__ __forceinline__ float2 mul_i(float2 v, int sgn) {
  return sgn > 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}
constexpr float kHalfSqrt3 = 0.86602540378443864676f;   // sin(2 pi / 3)

// v * exp(sgn 2 pi i j / n) for n in {1, 2, 3, 4}; with n, j, sgn constants after
// unrolling every branch folds away
__device__ __forceinline__ float2 twiddle(float2 v, int n, int j, int sgn) {
  j %= n;
  if (j == 0) return v;
  if (2 * j == n) return make_float2(-v.x, -v.y);
  if (4 * j == n) return mul_i(v, sgn);
  if (4 * j == 3 * n) return mul_i(v, -sgn);
  const float s = (j == 1 ? sgn : -sgn) * kHalfSqrt3;   // n == 3: cos = -1/2
  return make_float2(-0.5f * v.x - s * v.y, -0.5f * v.y + s * v.x);
}

// in-place length-N DFT with exponent sign sgn of x[o], x[o + st], ...
template <int N>
__device__ __forceinline__ void dft1(float2 *x, int o, int st, int sgn) {
  if (N == 2) {
    const float2 a = x[o], b = x[o + st];
    x[o] = cadd(a, b);
    x[o + st] = csub(a, b);
  } else if (N == 3) {
    const float2 a = x[o], b = x[o + st], c = x[o + 2 * st];
    const float2 t = cadd(b, c), d = csub(b, c);
    const float2 m = make_float2(a.x - 0.5f * t.x, a.y - 0.5f * t.y);
    const float2 s = make_float2(sgn * kHalfSqrt3 * d.x, sgn * kHalfSqrt3 * d.y);
    x[o] = cadd(a, t);
    x[o + st] = cadd(m, mul_i(s, 1));
    x[o + 2 * st] = csub(m, mul_i(s, 1));
  } else if (N == 4) {
    const float2 a = x[o], b = x[o + st], c = x[o + 2 * st], d = x[o + 3 * st];
    const float2 s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), w = mul_i(csub(b, d), sgn);
    x[o] = cadd(s0, s1);
    x[o + st] = cadd(d0, w);
    x[o + 2 * st] = csub(s0, s1);
    x[o + 3 * st] = csub(d0, w);
  }
}

// 2-D DFT over the (N2, N3) slab x[a * N3 + b]
template <int N2, int N3>
__device__ __forceinline__ void dft2(float2 (&x)[N2 * N3], int sgn) {
#pragma unroll
  for (int a = 0; a < N2; ++a) dft1<N3>(x, a * N3, 1, sgn);
#pragma unroll
  for (int b = 0; b < N3; ++b) dft1<N2>(x, b, N3, sgn);
}

// 16-byte asynchronous copy global -> shared (L2 only); bytes < 16 zero-fills the rest
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// slab m1 of b^+ and c^- at one k_s, from the staged planes (b: q = (x1, r) rows 0..NK-1,
// c: k_w rows NK..2NK-1, each EB elements apart), accumulated into acc
template <int N1, int N2, int N3, int EB, int M1>
__device__ __forceinline__ void dfft_step(const float2 *st, float2 (&acc)[N2 * N3]) {
  constexpr int P = N2 * N3, NK = N1 * P;
  float2 bt[P], ct[P];
#pragma unroll
  for (int x1 = 0; x1 < N1; ++x1)
#pragma unroll
    for (int r = 0; r < P; ++r) {
      const float2 v = st[(x1 * P + r) * EB], w = st[(NK + x1 * P + r) * EB];
      bt[r] = x1 == 0 ? v : cadd(bt[r], twiddle(v, N1, M1 * x1, 1));
      ct[r] = x1 == 0 ? w : cadd(ct[r], twiddle(w, N1, M1 * x1, -1));
    }
  dft2<N2, N3>(bt, 1);
  dft2<N2, N3>(ct, -1);
#pragma unroll
  for (int r = 0; r < P; ++r) {
    acc[r].x = fmaf(ct[r].x, bt[r].x, fmaf(-ct[r].y, bt[r].y, acc[r].x));
    acc[r].y = fmaf(ct[r].x, bt[r].y, fmaf(ct[r].y, bt[r].x, acc[r].y));
  }
}

// slab k1 of D: the inverse side-N1 transform of the exchanged (m1, k') values
template <int N1, int N2, int N3, int EB, int K1>
__device__ __forceinline__ void dfft_out(const float2 *s_x, int el, float inv_nk, double2 *Dk, long long NN) {
  constexpr int P = N2 * N3;
#pragma unroll
  for (int r = 0; r < P; ++r) {
    float2 s = s_x[r * EB + el];
#pragma unroll
    for (int m1 = 1; m1 < N1; ++m1) s = cadd(s, twiddle(s_x[(m1 * P + r) * EB + el], N1, m1 * K1, 1));
    double2 *d = Dk + (long long)(K1 * P + r) * NN;
    double2 v = *d;
    v.x += (double)(s.x * inv_nk);
    v.y += (double)(s.y * inv_nk);
    *d = v;
  }
}

template <int N1, int N2, int N3, int EB, int M1 = 0>
__device__ __forceinline__ void dfft_step_at(int m1, const float2 *st, float2 (&acc)[N2 * N3]) {
  if constexpr (M1 < N1) {
    if (m1 == M1)
      dfft_step<N1, N2, N3, EB, M1>(st, acc);
    else
      dfft_step_at<N1, N2, N3, EB, M1 + 1>(m1, st, acc);
  }
}

template <int N1, int N2, int N3, int EB, int K1 = 0>
__device__ __forceinline__ void dfft_out_at(int k1, const float2 *s_x, int el, float inv_nk, double2 *Dk, long long NN) {
  if constexpr (K1 < N1) {
    if (k1 == K1)
      dfft_out<N1, N2, N3, EB, K1>(s_x, el, inv_nk, Dk, NN);
    else
      dfft_out_at<N1, N2, N3, EB, K1 + 1>(k1, s_x, el, inv_nk, Dk, NN);
  }
}

template <int N1, int N2, int N3, int R, int S>
struct DfftShape {
  static constexpr int P = N2 * N3, NK = N1 * P, EB = 32 * R, NT = 32 * N1 * R;
  static constexpr size_t stage_elems = (size_t)2 * NK * EB;   // float2: NK b planes, NK c planes
  static constexpr size_t smem = S * stage_elems * sizeof(float2) + ((NK * NK + 15) / 16) * 16;
};

// Block: EB = 32 R elements x N1 slabs (warp w: slab w % N1, element group w / N1).  The
// 2 NK planes of one k_s (b: B[(q, k_s)], c: C[(k_w - k_s, k_w)]) are staged for the block
// by 16-byte asynchronous copies, S - 1 steps of k_s ahead of the arithmetic.
// Requires B, C 16-byte aligned and sP, sI, NN even (checked by the launcher).
template <int N1, int N2, int N3, int R, int S>
__global__ void __launch_bounds__(32 * N1 * R) k_kpoint_D_fft(const float2 *B, const float2 *C, long long sP,
                                                             long long sI, const int *sub, long long NN, int i0,
                                                             long long sDi, double2 *D) {
  using Sh = DfftShape<N1, N2, N3, R, S>;
  constexpr int P = Sh::P, NK = Sh::NK, EB = Sh::EB, NT = Sh::NT, CH = EB / 2;
  extern __shared__ __align__(16) unsigned char dsm[];
  float2 *buf = reinterpret_cast<float2 *>(dsm);
  unsigned char *s_sub = dsm + S * Sh::stage_elems * sizeof(float2);   // [k_w][k_s] -> k_w - k_s
  const int tid = threadIdx.x + 32 * threadIdx.y;
  for (int t = tid; t < NK * NK; t += NT) s_sub[t] = (unsigned char)sub[t];
  __syncthreads();
  const int il = blockIdx.y;
  const long long e0 = (long long)blockIdx.x * EB, rem = NN - e0;
  const float2 *Bb = B + (long long)il * sI + e0, *Cb = C + (long long)il * sI + e0;
  auto issue = [&](int ks) {
    float2 *dst = buf + (size_t)(ks % S) * Sh::stage_elems;
#pragma unroll 4
    for (int c = tid; c < 2 * NK * CH; c += NT) {
      const int j = c / CH, u = c % CH;
      const float2 *src = j < NK ? Bb + (long long)(j * NK + ks) * sP
                                 : Cb + (long long)(s_sub[(j - NK) * NK + ks] * NK + (j - NK)) * sP;
      const long long off = 2LL * u;
      const int bytes = off + 1 < rem ? 16 : (off < rem ? 8 : 0);
      cp_async16(dst + j * EB + 2 * u, bytes ? src + off : src, bytes);
    }
  };
#pragma unroll 1
  for (int st = 0; st < S - 1; ++st) {
    if (st < NK) issue(st);
    cp_async_commit();
  }
  const int m1 = threadIdx.y % N1, el = (threadIdx.y / N1) * 32 + threadIdx.x;
  float2 acc[P];
#pragma unroll
  for (int r = 0; r < P; ++r) acc[r] = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int ks = 0; ks < NK; ++ks) {
    cp_async_wait<S - 2>();   // this thread's copies of step ks have landed
    __syncthreads();          // everyone's have, and step ks - 1's slot is free
    if (ks + S - 1 < NK) issue(ks + S - 1);
    cp_async_commit();
    dfft_step_at<N1, N2, N3, EB>(m1, buf + (size_t)(ks % S) * Sh::stage_elems + el, acc);
  }
  cp_async_wait<0>();
  __syncthreads();
  dft2<N2, N3>(acc, 1);
#pragma unroll
  for (int r = 0; r < P; ++r) buf[(m1 * P + r) * EB + el] = acc[r];
  __syncthreads();
  if (el < rem)
    dfft_out_at<N1, N2, N3, EB>(m1, buf, el, 1.f / (float)NK, D + (long long)(i0 + il) * sDi + e0 + el, NN);
}

template <int N1, int N2, int N3, int R, int S>
cudaError_t launch_dfft(const float2 *B, const float2 *C, long long sP, long long sI, const int *sub, long long NN,
                        int ct, int i0, long long sDi, double2 *D, cudaStream_t s) {
  using Sh = DfftShape<N1, N2, N3, R, S>;
  static std::atomic<unsigned long long> attr{0};
  const cudaError_t e = set_smem_once(k_kpoint_D_fft<N1, N2, N3, R, S>, (int)Sh::smem, attr);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((NN + Sh::EB - 1) / Sh::EB), (unsigned)ct), block(32, N1 * R);
  k_kpoint_D_fft<N1, N2, N3, R, S><<<grid, block, Sh::smem, s>>>(B, C, sP, sI, sub, NN, i0, sDi, D);
  return cudaGetLastError();
}

// Split of rows that are contiguous in memory with K strided (a transposed read):
// a block stages a tile of RB rows x K in shared memory with coalesced loads, then one
// warp per row finds its scale and writes the FP16 pairs.  kind 0: A rows, 1: B rows.
constexpr int kRB = 32;
template <class T>
__global__ void __launch_bounds__(256) k_csplit_t(const T *src, RowMap m, int batch, int rows, int K, int Kp2, int kind,
                                                 float sa, float sbc, __half *hi, __half *lo, float *unscale) {
  extern __shared__ __align__(16) unsigned char tile_raw[];
  T *tile = reinterpret_cast<T *>(tile_raw);   // [K][kRB + 1]
  const int nrb = (rows + kRB - 1) / kRB;
  const int b = blockIdx.x / nrb, r0 = (blockIdx.x % nrb) * kRB;
  if (b >= batch) return;
  for (int idx = threadIdx.x; idx < K * kRB; idx += blockDim.x) {
    const int k = idx / kRB, rr = idx % kRB;
    T v{};
    if (r0 + rr < rows) v = src[m.row(b, r0 + rr) + k * m.sk];
    tile[k * (kRB + 1) + rr] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int rr = warp; rr < kRB; rr += 8) {
    const int r = r0 + rr;
    if (r >= rows) break;
    float mx = 0.f;
    for (int k = lane; k < K; k += 32) {
      const T v = tile[k * (kRB + 1) + rr];
      mx = fmaxf(mx, fmaxf((float)fabs(v.x), (float)fabs(v.y)));
    }
    mx = cwarp_max(mx);
    const float s = tc::pow2_floor_inv(mx);
    // lane pairs share a complex element (conflict-free tile reads); half2 stores
    if (kind == 0) {
      const long long row = (long long)b * rows + r;
      __half2 *h = reinterpret_cast<__half2 *>(hi + row * Kp2), *l = reinterpret_cast<__half2 *>(lo + row * Kp2);
      for (int k = lane; k < Kp2 / 2; k += 32) {
        __half a0 = __float2half(0.f), d0 = a0, a1 = a0, d1 = a0;
        if (k < K) {
          const T v = tile[k * (kRB + 1) + rr];
          split_pair(v.x, s, a0, d0);
          split_pair(v.y, s, a1, d1);
        }
        h[k] = __halves2half2(a0, a1);
        l[k] = __halves2half2(d0, d1);
      }
      if (lane == 0) unscale[row] = 1.f / s;
    } else {
      const long long row = ((long long)b * rows + r) * 2;
      __half2 *h0 = reinterpret_cast<__half2 *>(hi + row * Kp2), *l0 = reinterpret_cast<__half2 *>(lo + row * Kp2);
      __half2 *h1 = h0 + Kp2 / 2, *l1 = l0 + Kp2 / 2;
      for (int k = lane; k < Kp2 / 2; k += 32) {
        __half a0 = __float2half(0.f), d0 = a0, a1 = a0, d1 = a0, a2 = a0, d2 = a0, a3 = a0, d3 = a0;
        if (k < K) {
          const T v = tile[k * (kRB + 1) + rr];
          __half yh, yl;
          split_pair(v.x, s, a0, d0);
          split_pair(v.y, s, yh, yl);
          const bool n_re = sa * sbc > 0.f, n_im = sbc < 0.f, n_x = sa < 0.f;
          a1 = neg_if(n_re, yh);
          d1 = neg_if(n_re, yl);
          a2 = neg_if(n_im, yh);
          d2 = neg_if(n_im, yl);
          a3 = neg_if(n_x, a0);
          d3 = neg_if(n_x, d0);
        }
        h0[k] = __halves2half2(a0, a1);
        l0[k] = __halves2half2(d0, d1);
        h1[k] = __halves2half2(a2, a3);
        l1[k] = __halves2half2(d2, d3);
      }
      if (lane == 0) unscale[row] = unscale[row + 1] = 1.f / s;
    }
  }
}

// rows contiguous along the row index and K strided: stage through shared memory
template <class T>
bool launch_split_t(const T *src, const RowMap &m, int batch, int rows, int K, int Kp2, int kind, float sa, float sbc,
                    __half *hi, __half *lo, float *unscale, cudaStream_t s) {
  const bool contiguous = (m.R2 == 1 ? m.sr1 == 1 : m.sr2 == 1);
  if (!contiguous || m.sk == 1) return false;
  const size_t smem = (size_t)K * (kRB + 1) * sizeof(T);
  if (smem > 200 * 1024) return false;
  static std::atomic<unsigned long long> attr{0};
  if (set_smem_once(k_csplit_t<T>, 200 * 1024, attr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const long long blocks = (long long)batch * ((rows + kRB - 1) / kRB);
  k_csplit_t<T><<<(unsigned)blocks, 256, smem, s>>>(src, m, batch, rows, K, Kp2, kind, sa, sbc, hi, lo, unscale);
  return true;
}

// ----------------------------- real operands -----------------------------
__device__ __forceinline__ double ld_r(const double *p) { return *p; }
__device__ __forceinline__ float ld_r(const float *p) { return *p; }

template <class R>
__device__ __forceinline__ void store8_r(const R *v, float s, __half *h, __half *l) {
  uint32_t ph[4], pl[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    __half a0, d0, a1, d1;
    split_pair(v[2 * j], s, a0, d0);
    split_pair(v[2 * j + 1], s, a1, d1);
    ph[j] = pack_h2(a0, a1);
    pl[j] = pack_h2(d0, d1);
  }
  *reinterpret_cast<uint4 *>(h) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
  *reinterpret_cast<uint4 *>(l) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
}

// Real rows with K contiguous or strided: LPR lanes per row, 16-byte stores.
template <class T>
__global__ void k_rsplit(const T *src, const float *mul, RowMap m, int batch, int rows, int K, int Kp, __half *hi,
                         __half *lo, float *unscale) {
  const int lpr = lanes_per_row(Kp);
  const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gr = gt / lpr;
  const int gl = (int)(gt % lpr);
  const bool live = gr < (long long)rows * batch;
  const int b = live ? (int)(gr / rows) : 0, r = live ? (int)(gr % rows) : 0;
  const T *x = src + m.row(b, r);
  const float *mu = mul ? mul + m.row(0, r) : nullptr;
  auto val = [&](int k) -> T { return mu ? ld_r(x + k * m.sk) * static_cast<T>(mu[k * m.sk]) : ld_r(x + k * m.sk); };
  float mx = 0.f;
  if (live)
    for (int k = gl; k < K; k += lpr) mx = fmaxf(mx, (float)fabs(val(k)));
  mx = group_max(mx, lpr);
  if (!live) return;
  const float s = tc::pow2_floor_inv(mx);
  __half *h = hi + gr * Kp, *l = lo + gr * Kp;
  for (int c8 = gl; c8 < Kp / 8; c8 += lpr) {
    T v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = c8 * 8 + j;
      v[j] = k < K ? val(k) : T(0);
    }
    store8_r(v, s, h + c8 * 8, l + c8 * 8);
  }
  if (gl == 0) unscale[gr] = 1.f / s;
}

// Real rows contiguous along the row index with K strided: 32 rows per block, K in
// chunks of 64 through a shared-memory tile, twice (row maxima, then the FP16 pairs).
template <class T>
__global__ void __launch_bounds__(256) k_rsplit_t(const T *src, const float *mul, RowMap m, int batch, int rows, int K,
                                                 int Kp, __half *hi, __half *lo, float *unscale) {
  __shared__ T tile[64][kRB + 1];
  __shared__ float rmax[kRB];
  const int nrb = (rows + kRB - 1) / kRB;
  const int b = blockIdx.x / nrb, r0 = (blockIdx.x % nrb) * kRB;
  if (b >= batch) return;
  const int t = threadIdx.x;
  if (t < kRB) rmax[t] = 0.f;
  const int rr = t / 8, part = t % 8;   // phase 2: 8 threads per row, 8 values each
  float my = 0.f;
  for (int k0 = 0; k0 < K; k0 += 64) {
    __syncthreads();
    for (int idx = t; idx < 64 * kRB; idx += blockDim.x) {
      const int k = idx / kRB, c = idx % kRB;
      T v{};
      if (r0 + c < rows && k0 + k < K) {
        const long long off = m.row(0, r0 + c) + (long long)(k0 + k) * m.sk;
        v = src[(long long)b * m.sb + off];
        if (mul) v = v * static_cast<T>(mul[off]);
      }
      tile[k][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 8; ++j) my = fmaxf(my, fabsf((float)tile[part * 8 + j][rr]));
  }
  // row maxima: the 8 threads of a row are consecutive lanes
  for (int o = 4; o > 0; o >>= 1) my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
  const float sc = tc::pow2_floor_inv(my);
  const int r = r0 + rr;
  const long long row = (long long)b * rows + r;
  for (int k0 = 0; k0 < Kp; k0 += 64) {
    __syncthreads();
    for (int idx = t; idx < 64 * kRB; idx += blockDim.x) {
      const int k = idx / kRB, c = idx % kRB;
      T v{};
      if (r0 + c < rows && k0 + k < K) {
        const long long off = m.row(0, r0 + c) + (long long)(k0 + k) * m.sk;
        v = src[(long long)b * m.sb + off];
        if (mul) v = v * static_cast<T>(mul[off]);
      }
      tile[k][c] = v;
    }
    __syncthreads();
    if (r < rows) {
      T v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = tile[part * 8 + j][rr];
      store8_r(v, sc, hi + row * Kp + k0 + part * 8, lo + row * Kp + k0 + part * 8);
    }
  }
  if (r < rows && part == 0) unscale[row] = 1.f / sc;
  (void)rmax;
}

// FP32 rows with K contiguous and 16-byte aligned: one warp per row reads the row once
// into registers (16-byte loads, CH float4 per lane), finds its scale and writes the pairs.
// Requires the row storage to extend to a multiple of 4 floats (masked beyond K).
template <int CH>
__global__ void __launch_bounds__(256) k_rsplit_f32v(const float *src, const float *mul, RowMap m, int batch, int rows,
                                                    int K, int Kp, __half *hi, __half *lo, float *unscale) {
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (gw >= (long long)rows * batch) return;
  const int b = (int)(gw / rows), r = (int)(gw % rows);
  const long long roff = m.row(0, r);
  const float4 *x = reinterpret_cast<const float4 *>(src + (long long)b * m.sb + roff);
  const float4 *mu = mul ? reinterpret_cast<const float4 *>(mul + roff) : nullptr;
  float4 v[CH];
  float mx = 0.f;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int k4 = c * 32 + lane;
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k4 * 4 < K) {
      t = __ldg(x + k4);
      if (mu) {
        const float4 u = __ldg(mu + k4);
        t.x *= u.x; t.y *= u.y; t.z *= u.z; t.w *= u.w;
      }
      if (k4 * 4 + 1 >= K) t.y = 0.f;
      if (k4 * 4 + 2 >= K) t.z = 0.f;
      if (k4 * 4 + 3 >= K) t.w = 0.f;
    }
    v[c] = t;
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(t.x), fabsf(t.y)), fmaxf(fabsf(t.z), fabsf(t.w))));
  }
  mx = cwarp_max(mx);
  const float s = tc::pow2_floor_inv(mx);
  __half *h = hi + gw * Kp, *l = lo + gw * Kp;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int k4 = c * 32 + lane;
    if (k4 * 4 >= Kp) break;
    __half a[4], d[4];
    split_pair(v[c].x, s, a[0], d[0]);
    split_pair(v[c].y, s, a[1], d[1]);
    split_pair(v[c].z, s, a[2], d[2]);
    split_pair(v[c].w, s, a[3], d[3]);
    *reinterpret_cast<uint2 *>(h + k4 * 4) = make_uint2(pack_h2(a[0], a[1]), pack_h2(a[2], a[3]));
    *reinterpret_cast<uint2 *>(l + k4 * 4) = make_uint2(pack_h2(d[0], d[1]), pack_h2(d[2], d[3]));
  }
  if (lane == 0) unscale[gw] = 1.f / s;
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
  if (f32 ? launch_split_t(static_cast<const float2 *>(src), m, batch, rows, K, out.Kp2, 0, 1.f, 1.f, out.hi, out.lo,
                           out.unscale, s)
          : launch_split_t(static_cast<const double2 *>(src), m, batch, rows, K, out.Kp2, 0, 1.f, 1.f, out.hi, out.lo,
                           out.unscale, s))
    return;
  const int lpr = lanes_per_row(out.Kp2);
  const int blocks = (int)std::max<long long>(1, ((long long)rows * batch * lpr + 255) / 256);
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
  const float sa = conjA ? -1.f : 1.f, sbc = conjB ? -1.f : 1.f;
  if (f32 ? launch_split_t(static_cast<const float2 *>(src), m, batch, cols, K, out.Kp2, 1, sa, sbc, out.hi, out.lo,
                           out.unscale, s)
          : launch_split_t(static_cast<const double2 *>(src), m, batch, cols, K, out.Kp2, 1, sa, sbc, out.hi, out.lo,
                           out.unscale, s))
    return;
  const int lpr = lanes_per_row(out.Kp2);
  const int blocks = (int)std::max<long long>(1, ((long long)cols * batch * lpr + 255) / 256);
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

// The tensor core truncates its FP32 accumulator at every MMA step, a bias that grows with
// the number of steps; K beyond kKChunk is therefore split into windows whose partial
// products are added to C by the epilogue in round-to-nearest FP32.
constexpr int kKChunk = 1024;

Status cgemm_tc(sox_handle h, const CSplit &A, const CSplit &B, int batch, const int *idxA, const int *idxB,
                float alpha, float *C, long long ldc, long long sCb, cudaStream_t s, bool accumulate) {
  if (batch <= 0 || A.rows <= 0 || B.rows <= 0) return Status::ok();
  if (A.Kp2 != B.Kp2) return {SOX_ERR_INVALID_ARG, "cgemm_tc: operands split with different K"};
  if ((ldc & 3) || (sCb & 3) || (reinterpret_cast<uintptr_t>(C) & 15))
    return {SOX_ERR_INVALID_ARG, "cgemm_tc: output not 16-byte aligned"};
  const long long bsA = A.bstride ? A.bstride : A.rows, bsB = B.bstride ? B.bstride : B.rows;
  for (int k0 = 0; k0 < A.Kp2; k0 += kKChunk) {
    const int kw = std::min(kKChunk, A.Kp2 - k0);
    CUtensorMap maps[6];
    std::string err;
    if (!make_tmap_f16_3d_rs(&maps[0], A.hi + k0, kw, A.Kp2, A.rows, A.batch, bsA * A.Kp2, 64, 128, &err) ||
        !make_tmap_f16_3d_rs(&maps[1], A.lo + k0, kw, A.Kp2, A.rows, A.batch, bsA * A.Kp2, 64, 128, &err) ||
        !make_tmap_f16_3d_rs(&maps[2], B.hi + k0, kw, B.Kp2, B.rows, B.batch, bsB * B.Kp2, 64, 128, &err) ||
        !make_tmap_f16_3d_rs(&maps[3], B.lo + k0, kw, B.Kp2, B.rows, B.batch, bsB * B.Kp2, 64, 128, &err))
      return {SOX_ERR_CUDA, "cgemm_tc: " + err};
    if (!make_tmap_f32_store3d(&maps[4], C, B.rows, A.rows, batch, ldc, sCb, &err))
      return {SOX_ERR_CUDA, "cgemm_tc: " + err};
    maps[5] = maps[4];
    GemmTcArgs ga;
    ga.M = A.rows;
    ga.Ncols = B.rows;
    ga.Kp = kw;
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
    ga.accumulate = (accumulate || k0 > 0) ? 1 : 0;
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
  }
  return Status::ok();
}

Status kpoint_D_f32(const float *B, const float *C, long long sP, long long sI, const int *add, const int *sub,
                    const int mesh[3], long long NN, int ct, int i0, long long sDi, double *D, cudaStream_t s) {
  const int nk = mesh[0] * mesh[1] * mesh[2];
  // mesh sides up to 4: the Fourier form (n_k^2 products per element), 16-byte staged copies
  const bool aligned16 = ((reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15) == 0 &&
                         (sP % 2) == 0 && (sI % 2) == 0 && (NN % 2) == 0;
  if (aligned16) {
    const float2 *Bf = reinterpret_cast<const float2 *>(B), *Cf = reinterpret_cast<const float2 *>(C);
    double2 *Dd = reinterpret_cast<double2 *>(D);
    const int key = mesh[0] * 100 + mesh[1] * 10 + mesh[2];
    bool done = true;
    switch (key) {
#define SOX_DFFT(A, B_, C_, R, S)                                                              \
  case A * 100 + B_ * 10 + C_:                                                                \
    SOX_CUDA_TRY((launch_dfft<A, B_, C_, R, S>(Bf, Cf, sP, sI, sub, NN, ct, i0, sDi, Dd, s))); \
    break;
      SOX_DFFT(1, 1, 1, 4, 3) SOX_DFFT(1, 1, 2, 4, 3) SOX_DFFT(1, 2, 1, 4, 3) SOX_DFFT(2, 1, 1, 2, 3)
      SOX_DFFT(1, 1, 3, 4, 3) SOX_DFFT(1, 3, 1, 4, 3) SOX_DFFT(3, 1, 1, 1, 3) SOX_DFFT(1, 2, 2, 4, 3)
      SOX_DFFT(2, 2, 1, 2, 3) SOX_DFFT(2, 1, 2, 2, 3) SOX_DFFT(2, 2, 2, 2, 3) SOX_DFFT(3, 3, 1, 1, 3)
      SOX_DFFT(3, 3, 3, 1, 3) SOX_DFFT(1, 1, 4, 4, 3) SOX_DFFT(4, 1, 1, 1, 3) SOX_DFFT(2, 2, 4, 2, 2)
      SOX_DFFT(4, 4, 4, 1, 2)
#undef SOX_DFFT
      default:
        done = false;
    }
    if (done) return Status::ok();
  }
  {
    dim3 grid((unsigned)((NN + 127) / 128), (unsigned)ct);
    const float2 *Bf = reinterpret_cast<const float2 *>(B), *Cf = reinterpret_cast<const float2 *>(C);
    double2 *Dd = reinterpret_cast<double2 *>(D);
    bool done = true;
    switch (nk) {
#define SOX_DREG(K)                                                                      \
  case K:                                                                               \
    k_kpoint_D_reg<K><<<grid, 128, 0, s>>>(Bf, Cf, sP, sI, add, sub, NN, i0, sDi, Dd); \
    break;
      SOX_DREG(1) SOX_DREG(2) SOX_DREG(3) SOX_DREG(4) SOX_DREG(5) SOX_DREG(6) SOX_DREG(8) SOX_DREG(9)
      SOX_DREG(12) SOX_DREG(16) SOX_DREG(18) SOX_DREG(27) SOX_DREG(32) SOX_DREG(36) SOX_DREG(48) SOX_DREG(64)
#undef SOX_DREG
      default:
        done = false;
    }
    if (done) {
      SOX_CUDA_TRY(cudaGetLastError());
      return Status::ok();
    }
  }
  const long long np = (long long)nk * nk;
  const size_t per_e = (size_t)np * 2 * sizeof(float2);
  const size_t cap = 96 * 1024;
  if (per_e > cap) return {SOX_ERR_SHAPE, "k-mesh too large for the split-precision D step"};
  const int E = (int)std::min<size_t>(8, cap / per_e);
  static std::atomic<unsigned long long> attr{0};
  SOX_CUDA_TRY(set_smem_once(k_kpoint_D_blk, (int)cap, attr));
  dim3 grid((unsigned)((NN + E - 1) / E), (unsigned)ct);
  k_kpoint_D_blk<<<grid, 256, per_e * E, s>>>(reinterpret_cast<const float2 *>(B), reinterpret_cast<const float2 *>(C),
                                              sP, sI, add, sub, nk, NN, E, i0, sDi, reinterpret_cast<double2 *>(D));
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

int rsplit_kp(int K) { return ((K + 63) / 64) * 64; }

size_t rsplit_bytes(int batch, int rows, int K) {
  const size_t e = (size_t)batch * rows * rsplit_kp(K);
  return 2 * aligned_bytes(e, 2) + aligned_bytes((size_t)batch * rows, 4);
}

CSplit rsplit_take(Arena &ar, int batch, int rows, int K) {
  CSplit c;
  c.batch = batch;
  c.rows = rows;
  c.Kp2 = rsplit_kp(K);
  const size_t e = (size_t)batch * rows * c.Kp2;
  c.hi = ar.take<__half>(e);
  c.lo = ar.take<__half>(e);
  c.unscale = ar.take<float>((size_t)batch * rows);
  if (!c.unscale) c.hi = nullptr;
  return c;
}

void rsplit(const void *src, bool f32, long long sb, long long sr1, long long sr2, int R2, long long sk, int batch,
            int rows, int K, const CSplit &out, cudaStream_t s, const float *mul) {
  RowMap m{sb, sr1, sr2, sk, R2 > 0 ? R2 : 1};
  if (R2 <= 0) {
    m.sr2 = 0;
    m.R2 = 1;
  }
  const bool contiguous_rows = (m.R2 == 1 ? m.sr1 == 1 : m.sr2 == 1);
  if (contiguous_rows && sk != 1) {
    const long long blocks = (long long)batch * ((rows + kRB - 1) / kRB);
    if (f32)
      k_rsplit_t<float><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const float *>(src), mul, m, batch, rows, K,
                                                         out.Kp2, out.hi, out.lo, out.unscale);
    else
      k_rsplit_t<double><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const double *>(src), mul, m, batch, rows, K,
                                                          out.Kp2, out.hi, out.lo, out.unscale);
    return;
  }
  // FP32 rows, K contiguous, 16-byte aligned rows whose storage reaches a multiple of 4 floats
  const bool vec = f32 && sk == 1 && m.R2 == 1 && (m.sr1 % 4 == 0) && (m.sb % 4 == 0) && m.sr1 >= ((K + 3) & ~3) &&
                   (reinterpret_cast<uintptr_t>(src) % 16 == 0) && (!mul || reinterpret_cast<uintptr_t>(mul) % 16 == 0) &&
                   out.Kp2 <= 2048;
  if (vec) {
    const int blocks = (int)std::max<long long>(1, ((long long)rows * batch * 32 + 255) / 256);
    const float *fs = static_cast<const float *>(src);
    const int ch = (out.Kp2 + 127) / 128;
    if (ch <= 1)
      k_rsplit_f32v<1><<<blocks, 256, 0, s>>>(fs, mul, m, batch, rows, K, out.Kp2, out.hi, out.lo, out.unscale);
    else if (ch <= 2)
      k_rsplit_f32v<2><<<blocks, 256, 0, s>>>(fs, mul, m, batch, rows, K, out.Kp2, out.hi, out.lo, out.unscale);
    else if (ch <= 4)
      k_rsplit_f32v<4><<<blocks, 256, 0, s>>>(fs, mul, m, batch, rows, K, out.Kp2, out.hi, out.lo, out.unscale);
    else if (ch <= 8)
      k_rsplit_f32v<8><<<blocks, 256, 0, s>>>(fs, mul, m, batch, rows, K, out.Kp2, out.hi, out.lo, out.unscale);
    else
      k_rsplit_f32v<16><<<blocks, 256, 0, s>>>(fs, mul, m, batch, rows, K, out.Kp2, out.hi, out.lo, out.unscale);
    return;
  }
  const int lpr = lanes_per_row(out.Kp2);
  const int blocks = (int)std::max<long long>(1, ((long long)rows * batch * lpr + 255) / 256);
  if (f32)
    k_rsplit<float><<<blocks, 256, 0, s>>>(static_cast<const float *>(src), mul, m, batch, rows, K, out.Kp2, out.hi,
                                           out.lo, out.unscale);
  else
    k_rsplit<double><<<blocks, 256, 0, s>>>(static_cast<const double *>(src), mul, m, batch, rows, K, out.Kp2, out.hi,
                                            out.lo, out.unscale);
}

}  // namespace sox
