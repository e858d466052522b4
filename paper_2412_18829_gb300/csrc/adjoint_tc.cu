// Adjoint of Phi_SOX with respect to X and V in split precision (SOX_PREC_F16X2):
// the reverse pass of the FP64 form (adjoint.cu) on the tensor cores.
//
// Per spin and tau_j (c_j = -w_j dphi / 4), with A_v = U1 G(-tau_j)[:, v],
// B_v = A_v GR^T, C_v = GWt U2_v^T and E = X G(-tau_j) X^T:
//   Bbar_v = c_j E o C_v,  Cbar_v = c_j E o B_v,  Ebar = c_j sum_v B_v o C_v
//   Abar_v = Bbar_v GR,            GRbar = sum_v Bbar_v^T A_v,
//   GWtbar = sum_v Cbar_v U2_v,    U2bar_v += Cbar_v^T GWt,
//   U1bar += sum_v Abar_v (x) G(-tau_j)[:, v]
// then Xbar += GRbar G(tau_j)^T + GWtbar G(tau_j) - (Ebar X) G(-tau_j)^T - (Ebar^T X) G(-tau_j)
// (one split GEMM per chunk, accumulated in FP64), and at the end
//   Vbar = (U1bar + U2bar) Y^T,  Z = V^T (U1bar + U2bar),  Xbar += pair-product adjoint of Z.
// The projections G_Rq = X G(tau), G_wP^T = X G(tau)^T stay FP64, computed once per spin for
// every tau (E of tau_j reuses G_Rq of tau_{T-1-j}).
//
// B_v and C_v are never stored.  One fused kernel (k_adj_bc) recomputes them per
// 128 x 128 (P, R) tile in TMEM -- the forward's TMA / MMA pipeline -- and its epilogue
// forms Bbar_v and Cbar_v from E held in registers, writes them once as FP16 pairs
// [tau][v][R][P] (coalesced: a warp's lanes hold consecutive P) and accumulates Ebar.  The
// four reverse contractions then read those pairs in place: over R as K-major operands and over P as MN-major ones (gemm_mn.cu),
// so no transposed copy and no FP32 round trip of the n N^2 tensors exists.  Every split
// operand carries one power-of-two scale per tensor (per tau chunk), which is what lets
// one layout serve both contraction orders.
#include <algorithm>
#include <atomic>
#include <vector>

#include "adjoint.h"
#include "ctc.h"
#include "gemm_mn.h"
#include "smem_attr.h"
#include "tc_common.cuh"
#include "tc_kernels.h"

namespace sox {
namespace {

using tc::smem_u32;

long long rup4(long long x) { return (x + 3) & ~3LL; }
int rup(int x, int m) { return (x + m - 1) / m * m; }
int grid1(long long total) { return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 65535 * 8)); }

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
__global__ void k_to_f64(const float *in, long long ld, long long rows, int cols, double *out) {
  const long long total = rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (double)in[(e / cols) * ld + e % cols];
}

// out (FP64, rows x cols) += in (FP32, row length ld)
__global__ void k_add_f64(const float *in, long long ld, long long rows, int cols, double *out) {
  const long long total = rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    out[e] += (double)in[(e / cols) * ld + e % cols];
}

// dst[b] = src[b] (count values each) where flag[b] is set
__global__ void k_copy_flagged(const double *src, double *dst, long long count, int batch, const int *flag) {
  const long long total = count * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    if (flag[e / count]) dst[e] = src[e];
}

__global__ void k_fill(float *p, int count, float v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) p[i] = v;
}

// Scale bookkeeping of one tau chunk (device side: the maxima are device values).
//   in:  mx[0] = max |E| over the chunk (E = X G(-tau) X^T), sc[0..3] = scales of GR, GWt,
//        G(-tau) and U1 / U2 splits (one for both, the mixed tensor is split once), os the
//        A-GEMM's output scale.
//   out: f[0] = g (Bbar, Cbar storage scale), f[1..5] = output factors of the contractions
//        Abar, GRbar, GWtbar, U2bar, U1bar (the last completed once Abar's scale is known),
//        cg[b] = c_b g, em[b] = c_b / (sA sR sW sU)
struct AdjScalars {
  float mx[12];   // atomicMax targets: E, Abar, mixed tensor, X, G(-tau), GR, GWt, Ebar,
                  // the Xbar GEMM's A (projection adjoints) and B (G(tau), G(-tau)) operands
  float sc[12];   // scales: GR, GWt, G(-tau), U, Abar, X, Ebar, Xbar A, Xbar B
  float f[12];    // output factors of the contractions
};
constexpr int kFacG = 0, kFacAbar = 1, kFacGRbar = 2, kFacGWtbar = 3, kFacU2bar = 4, kFacU1bar = 5, kFacEX = 6,
              kFacXbar = 7;
constexpr int kScGR = 0, kScGW = 1, kScGm = 2, kScU = 3, kScAbar = 4, kScX = 5, kScEbar = 6, kScXa = 7, kScXb = 8;
constexpr int kMxXa = 8, kMxXb = 9;

__device__ __forceinline__ float pow2_floor(double x) {
  // largest power of two <= x (x > 0), clamped to normal FP32
  int e;
  frexp(x, &e);   // x = f 2^e, f in [0.5, 1)
  int k = e - 1;
  k = k < -126 ? -126 : (k > 126 ? 126 : k);
  return ldexpf(1.f, k);
}

__global__ void k_adj_factors(AdjScalars *sc, const double *w, const double *dphi, int j0, int bc, int n, float os,
                              float *cg, float *em) {
  if (blockIdx.x != 0) return;
  const double sR = sc->sc[kScGR], sW = sc->sc[kScGW], sG = sc->sc[kScGm], sU = sc->sc[kScU];
  const double sA = sU * sG * (double)os;
  double cmax = 0.0;
  for (int b = 0; b < bc; ++b) cmax = fmax(cmax, fabs(0.25 * w[j0 + b] * dphi[0]));
  const double bound = cmax * (double)sc->mx[0] * (double)n * 1073741824.0;   // |c E C~| <= c max|E| n 2^30
  const double g = bound > 0.0 ? (double)pow2_floor(32768.0 / bound) : 1.0;
  for (int b = threadIdx.x; b < bc; b += blockDim.x) {
    const double c = -0.25 * w[j0 + b] * dphi[0];
    cg[b] = (float)(c * g);
    em[b] = (float)(c / (sA * sR * sW * sU));
  }
  if (threadIdx.x == 0) {
    sc->f[kFacG] = (float)g;
    sc->f[kFacAbar] = (float)(1.0 / (g * sW * sU * sR));
    sc->f[kFacGRbar] = (float)(1.0 / (g * sW * sU * sA));
    sc->f[kFacGWtbar] = (float)(1.0 / (g * sA * sR * sU));
    sc->f[kFacU2bar] = (float)(1.0 / (g * sA * sR * sW));
  }
}

__global__ void k_u1bar_factor(AdjScalars *sc) {
  sc->f[kFacU1bar] = (float)(1.0 / ((double)sc->sc[kScAbar] * (double)sc->sc[kScGm]));
}

__global__ void k_ex_factor(AdjScalars *sc) {
  sc->f[kFacEX] = (float)(1.0 / ((double)sc->sc[kScEbar] * (double)sc->sc[kScX]));
}

__global__ void k_xbar_factor(AdjScalars *sc) {
  sc->f[kFacXbar] = (float)(1.0 / ((double)sc->sc[kScXa] * (double)sc->sc[kScXb]));
}

// ============================================================================
// Fused producer: for every (tau b, 128 x 128 (P, R) tile), over v,
//   B~_v = A~_v GR~^T, C~_v = GWt~ U2~_v^T in TMEM (double-buffered), and in the epilogue
//   Bbar_v = cg_b E o C~_v, Cbar_v = cg_b E o B~_v -> FP16 pairs [b][v][R][P],
//   Ebar  += B~_v o C~_v (registers), written em_b * sum at the end of the tile.
// Warp 0: TMA, warps 1 and 2: MMA (one thread each: the B_v and the C_v chunks), warps 4-11:
// pair writers, warps 12-19: Ebar accumulators (lane quarter warp % 4, column half by
// warpgroup).
// ============================================================================
constexpr int kT = 128, kC = 64;
constexpr int kTileB = kT * kC * 2;            // 16 KB: one 64-wide chunk of 128 rows, hi or lo
constexpr int kStageB = 4 * kTileB;
constexpr int kSt = 3;
// 20 warps: warpgroup 0 = TMA warp, MMA warp and two idle warps; warpgroups 1-2 write the
// pairs of columns [0, 64) and [64, 128) of the tile (E held in registers), warpgroups 3-4
// accumulate Ebar over the same halves.  Launched at 96 registers a thread (640 x 96 of the
// SM's 65536); warpgroup 0 gives registers back (kRegCtl) and the epilogue takes them
// (kRegEpi): 128 x kRegCtl + 512 x kRegEpi <= 640 x 96, the launch's own total (checked
// on the host against the compiled register count before the first launch).
constexpr int kProdThreads = 640, kProdEpi = 512;
constexpr int kRegLaunch = 96, kRegCtl = 56, kRegEpi = 104;
static_assert(128 * kRegCtl + 512 * kRegEpi <= kProdThreads * kRegLaunch, "register split above the launch total");

// full[q][s]: stage s holds a chunk for MMA issuer q (each issuer waits on its own set, so
// the phases it counts are the ones it consumes)
struct PBars {
  uint64_t full[2][kSt];
  uint64_t empty[kSt];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

struct AdjBcArgs {
  int n = 0, N = 0, Kp = 0, batch = 0;
  int v0 = 0, v1 = 0;             // the v sum runs over [v0, v1); outputs hold v - v0
  long long spin_limit = 0;
  int *status = nullptr;
  const float *E = nullptr;       // [b][N][ldE]
  long long ldE = 0, sE = 0;
  const float *cg = nullptr, *em = nullptr;   // [b]
  float *Ebar = nullptr;          // [b][N][ldE]
  __half *Bh = nullptr, *Bl = nullptr, *Ch = nullptr, *Cl = nullptr;   // [b][v][R][P], Rp x Rp
  long long Rp = 0;   // N rounded up to 128: rows R and row length P of the pairs
};

__device__ __forceinline__ long long wind_down(long long cap) { return cap > (1LL << 20) ? cap : (1LL << 20); }

// 3 x KS MMAs of one 64-wide K chunk (KS 16-wide steps; the last chunk of the n-long
// contraction stops at its first all-padding step)
template <int KS>
__device__ __forceinline__ void issue_split_ks(uint32_t acc, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                               uint32_t b_lo, bool first, uint32_t idesc) {
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const uint32_t off = k * 32;
    tc::mma_f16(acc, tc::desc_kmajor_sw128(a_hi + off), tc::desc_kmajor_sw128(b_lo + off), idesc,
                (first && k == 0) ? 0u : 1u);
    tc::mma_f16(acc, tc::desc_kmajor_sw128(a_lo + off), tc::desc_kmajor_sw128(b_hi + off), idesc, 1u);
  }
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const uint32_t off = k * 32;
    tc::mma_f16(acc, tc::desc_kmajor_sw128(a_hi + off), tc::desc_kmajor_sw128(b_hi + off), idesc, 1u);
  }
}
__device__ __forceinline__ void issue_split(uint32_t acc, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                            bool first, int ks, uint32_t idesc) {
  if (ks >= kC / 16) issue_split_ks<kC / 16>(acc, a_hi, a_lo, b_hi, b_lo, first, idesc);
  else if (ks == 3) issue_split_ks<3>(acc, a_hi, a_lo, b_hi, b_lo, first, idesc);
  else if (ks == 2) issue_split_ks<2>(acc, a_hi, a_lo, b_hi, b_lo, first, idesc);
  else issue_split_ks<1>(acc, a_hi, a_lo, b_hi, b_lo, first, idesc);
}

__device__ __forceinline__ uint32_t pack2(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// Columns c .. c+7 of E o y for this lane's row as FP16 pairs: lanes 2i and 2i+1 (rows P, P+1)
// swap halves so the even lane stores rows (P, P+1) of column c+2k and the odd lane those of
// column c+2k+1, each as one 4-byte word at dh / dl + column * Rp (P contiguous).
template <int NC>
__device__ __forceinline__ void store_pairs(const float (&e)[NC], int c, const float (&y)[8], __half *dh, __half *dl,
                                            long long Rp, bool even) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __half h0, l0, h1, l1;
    tc::split_f16(e[c + 2 * k] * y[2 * k], h0, l0);
    tc::split_f16(e[c + 2 * k + 1] * y[2 * k + 1], h1, l1);
    const uint32_t mh = pack2(h0, h1), ml = pack2(l0, l1);
    const uint32_t oh = __shfl_xor_sync(0xffffffffu, mh, 1), ol = __shfl_xor_sync(0xffffffffu, ml, 1);
    const long long col = (long long)(c + 2 * k + (even ? 0 : 1)) * Rp;
    *reinterpret_cast<uint32_t *>(dh + col) = even ? __byte_perm(mh, oh, 0x5410) : __byte_perm(oh, mh, 0x7632);
    *reinterpret_cast<uint32_t *>(dl + col) = even ? __byte_perm(ml, ol, 0x5410) : __byte_perm(ol, ml, 0x7632);
  }
}

// Epilogue of k_adj_bc for the NC columns [col0, col0 + NC) of every tile (lane quarter q):
// kWrite threads hold E and write the pairs, the others accumulate Ebar.  Both wait for every
// v's accumulators and hand them back.
template <int NC, bool kWrite>
__device__ __forceinline__ void adj_epilogue(PBars *bar, uint32_t tmem, const AdjBcArgs &a, int tP, long long total,
                                             volatile int *abort, int q, int lane, int col0) {
  const int tiles_per_b = tP * tP;
  const int row = q * 32 + lane;
  long long acc_it = 0;
  for (long long t = blockIdx.x; t < total && !*abort; t += gridDim.x) {
    const int b = (int)(t / tiles_per_b);
    const int r = (int)(t % tiles_per_b);
    const int P0 = (r / tP) * kT, R0 = (r % tP) * kT;
    const int P = P0 + row, Rh = R0 + col0;
    const bool prow = P < a.N;
    float x[NC];   // kWrite: E * c_b g; else: the Ebar accumulator
    if (kWrite) {
      const float cgb = a.cg[b];
      const float *Er = a.E + (long long)b * a.sE + (long long)(prow ? P : 0) * a.ldE;
#pragma unroll
      for (int j = 0; j < NC; ++j) x[j] = (prow && Rh + j < a.N) ? Er[Rh + j] * cgb : 0.f;
    } else {
#pragma unroll
      for (int j = 0; j < NC; ++j) x[j] = 0.f;
    }
    // pairs [b][v][R][P] (pitch Rp for both): lanes hold 32 consecutive P, and lane pairs swap
    // halves so each writes 4 bytes of two consecutive P of one column R
    const long long vstride = a.Rp * a.Rp;
    const int nv = a.v1 - a.v0;
    const bool even = (lane & 1) == 0;
    const int Pe = P0 + q * 32 + (lane & ~1);   // the even row of this lane's pair
    const long long obase = (long long)b * nv * vstride + (long long)Rh * a.Rp + Pe;
    bool ok = true;
    for (int v = a.v0; v < a.v1; ++v, ++acc_it) {
      const int buf = (int)(acc_it & 1);
      const uint32_t aph = (uint32_t)((acc_it >> 1) & 1);
      ok = tc::mbar_wait(&bar->acc_full[buf], aph, a.spin_limit, abort, a.status, 8);
      if (!ok) break;
      tc::tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + buf * 256 + col0;
      const long long o = obase + (v - a.v0) * vstride;
#pragma unroll
      for (int c = 0; c < NC; c += 8) {
        float bv[8], cv[8];
        tc::tmem_ld_32x32b_x8(base + c, bv);
        tc::tmem_ld_32x32b_x8(base + 128 + c, cv);
        tc::tmem_ld_wait();
        if (kWrite) {   // Bbar = E o C, then Cbar = E o B
          store_pairs<NC>(x, c, cv, a.Bh + o, a.Bl + o, a.Rp, even);
          store_pairs<NC>(x, c, bv, a.Ch + o, a.Cl + o, a.Rp, even);
        } else {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) x[c + jj] = fmaf(bv[jj], cv[jj], x[c + jj]);
        }
      }
      tc::tc_fence_before();
      tc::mbar_arrive(&bar->acc_empty[buf]);
    }
    if (!ok) break;
    if (!kWrite && prow) {
      const float emb = a.em[b];
      float *Eo = a.Ebar + (long long)b * a.sE + (long long)P * a.ldE;
#pragma unroll
      for (int j = 0; j < NC; ++j)
        if (Rh + j < a.N) Eo[Rh + j] = x[j] * emb;
    }
  }
}

__global__ void __launch_bounds__(kProdThreads, 1)
    k_adj_bc(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
             const __grid_constant__ CUtensorMap tmGR_hi, const __grid_constant__ CUtensorMap tmGR_lo,
             const __grid_constant__ CUtensorMap tmGW_hi, const __grid_constant__ CUtensorMap tmGW_lo,
             const __grid_constant__ CUtensorMap tmU_hi, const __grid_constant__ CUtensorMap tmU_lo, AdjBcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  PBars *bar = reinterpret_cast<PBars *>(smem + kSt * kStageB);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tP = (a.N + kT - 1) / kT;
  const int tiles_per_b = tP * tP;
  const long long total = (long long)a.batch * tiles_per_b;
  const int nk = a.Kp / kC;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kSt; ++s) {
      tc::mbar_init(&bar->full[0][s], 1);
      tc::mbar_init(&bar->full[1][s], 1);
      tc::mbar_init(&bar->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bar->acc_full[b], 2);   // one commit per issuing warp
      tc::mbar_init(&bar->acc_empty[b], kProdEpi);
    }
    tc::mbar_init(&bar->drain, 2);
    bar->abort = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(&bar->tmem_base, 512);
    tc::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmA_hi); tc::prefetch_tmap(&tmA_lo); tc::prefetch_tmap(&tmGR_hi);
    tc::prefetch_tmap(&tmGR_lo); tc::prefetch_tmap(&tmGW_hi); tc::prefetch_tmap(&tmGW_lo);
    tc::prefetch_tmap(&tmU_hi); tc::prefetch_tmap(&tmU_lo);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = bar->tmem_base;
  volatile int *abort = &bar->abort;
  if (warp >= 4) {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegEpi));
    const int grp = (warp - 4) >> 2;   // 0, 1: pair writers; 2, 3: Ebar
    if (grp < 2)
      adj_epilogue<64, true>(bar, tmem, a, tP, total, abort, warp & 3, lane, grp * 64);
    else
      adj_epilogue<64, false>(bar, tmem, a, tP, total, abort, warp & 3, lane, (grp - 2) * 64);
  } else {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegCtl));
  if (warp == 0) {
    if (lane == 0) {
      long long it = 0;
      tc::RingPhases ring;
      for (long long t = blockIdx.x; t < total && !*abort; t += gridDim.x) {
        const int b = (int)(t / tiles_per_b);
        const int r = (int)(t % tiles_per_b);
        const int P0 = (r / tP) * kT, R0 = (r % tP) * kT;
        for (int v = a.v0; v < a.v1 && !*abort; ++v) {
          for (int p = 0; p < 2 * nk && !*abort; ++p, ++it) {
            int kc, half;
            tc::bc_decode(p, nk, 1, kc, half);
            const int s = (int)(it % kSt);
            const uint32_t ph = (uint32_t)((it / kSt) & 1);
            if (!tc::mbar_wait(&bar->empty[s], ph ^ 1u, a.spin_limit, abort, a.status, 1)) break;
            uint64_t *fb = &bar->full[half][s];   // the half's issuer
            ring.take(half, s);
            tc::mbar_arrive_expect_tx(fb, kStageB);
            uint8_t *st = smem + (size_t)s * kStageB;
            const int x = kc * kC;
            if (half == 0) {   // B_v = A_v GR^T
              tc::tma_load_3d(st, &tmA_hi, fb, x, P0, b * a.n + v);
              tc::tma_load_3d(st + kTileB, &tmA_lo, fb, x, P0, b * a.n + v);
              tc::tma_load_3d(st + 2 * kTileB, &tmGR_hi, fb, x, R0, b);
              tc::tma_load_3d(st + 3 * kTileB, &tmGR_lo, fb, x, R0, b);
            } else {           // C_v = GWt U2_v^T
              tc::tma_load_3d(st, &tmGW_hi, fb, x, P0, b);
              tc::tma_load_3d(st + kTileB, &tmGW_lo, fb, x, P0, b);
              tc::tma_load_3d(st + 2 * kTileB, &tmU_hi, fb, x, R0, v);
              tc::tma_load_3d(st + 3 * kTileB, &tmU_lo, fb, x, R0, v);
            }
          }
        }
      }
      // every copy issued has landed before the CTA exits
      tc::ring_wind_down(bar->full, ring, wind_down(a.spin_limit));
    }
  } else if (warp == 1 || warp == 2) {
    // two MMA issuers, warp 1 the B_v chunks and warp 2 the C_v chunks (each into its own
    // accumulators; the producer alternates them in the ring): while one waits for a stage
    // the other keeps the tensor pipe fed
    if (lane == 0) {
      const int my = warp - 1;
      long long it = 0, acc_it = 0;
      tc::RingPhases ring;   // this issuer's phases on its set, full[my][.]
      bool ok = true;
      for (long long t = blockIdx.x; t < total && ok && !*abort; t += gridDim.x) {
        // N = the R tile's valid width rounded up to 16 (the last tile stops at N)
        const int R0 = (int)((t % tiles_per_b) % tP) * kT;
        const int wR = a.N - R0 >= kT ? kT : ((a.N - R0 + 15) & ~15);
        const uint32_t idesc = tc::idesc_f16_f32(kT, wR);
        for (int v = a.v0; v < a.v1 && ok; ++v, ++acc_it) {
          const int buf = (int)(acc_it & 1);
          const uint32_t aph = (uint32_t)((acc_it >> 1) & 1);
          ok = tc::mbar_wait(&bar->acc_empty[buf], aph ^ 1u, a.spin_limit, abort, a.status, 2);
          if (!ok) break;
          tc::tc_fence_after();
          {   // this issuer's chunks, at the ring positions bc_pos gives
            const int half = my;
            const uint32_t acc = tmem + buf * 256 + half * 128;
            for (int kc = 0; kc < nk; ++kc) {
              const int s = (int)((it + tc::bc_pos(kc, my, nk, 1)) % kSt);
              ok = tc::mbar_wait(&bar->full[my][s], ring.take(my, s), a.spin_limit, abort, a.status, 4);
              if (!ok) break;
              tc::tc_fence_after();
              const uint32_t st = smem_u32(smem + (size_t)s * kStageB);
              issue_split(acc, st, st + kTileB, st + 2 * kTileB, st + 3 * kTileB, kc == 0,
                          a.n - kc * kC >= kC ? kC / 16 : (a.n - kc * kC + 15) / 16, idesc);
              tc::mma_commit(&bar->empty[s]);
            }
          }
          it += 2 * nk;
          if (ok) tc::mma_commit(&bar->acc_full[buf]);
        }
      }
      tc::mma_commit(&bar->drain);   // all MMAs complete before TMEM is released
      for (long long i = 0; i < wind_down(a.spin_limit) && !tc::mbar_try_wait(&bar->drain, 0); ++i) {
      }
    }
  }
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

size_t adj_bc_smem() { return (size_t)kSt * kStageB + sizeof(PBars) + 1024; }

cudaError_t launch_adj_bc(const CUtensorMap *m, const AdjBcArgs &a, int grid, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  static std::atomic<int> regs_ok{0};
  if (regs_ok.load() == 0) {
    // the register split is sized for the launch's own allocation: refuse to launch if the
    // compiled kernel starts with fewer registers (the increase would never be granted)
    cudaFuncAttributes fa;
    const cudaError_t e0 = cudaFuncGetAttributes(&fa, k_adj_bc);
    if (e0 != cudaSuccess) return e0;
    if (fa.numRegs < kRegLaunch) return cudaErrorInvalidConfiguration;
    regs_ok.store(1);
  }
  const cudaError_t e = set_smem_once(k_adj_bc, (int)adj_bc_smem(), attr);
  if (e != cudaSuccess) return e;
  k_adj_bc<<<grid, kProdThreads, adj_bc_smem(), s>>>(m[0], m[1], m[2], m[3], m[4], m[5], m[6], m[7], a);
  return cudaGetLastError();
}

// ------------------------------- geometry ----------------------------------

struct AdjGeom {
  int n, N, T, S;
  int Kp;           // n padded to 64: K of the forward contractions, pitch of the splits
  int NR;           // P / R rows of the forward operands (>= 128)
  int RG;           // rows of G(-tau)^T per tau (>= 128)
  long long Rp;     // row pitch of Bbar / Cbar (N rounded up to 128)
  long long nn, np4, np8, nnp, ldN, ldN8, Nn;
  long long abar_pitch;   // per-v pitch of the Abar split [(P, q)] (N n rounded up to 8)
  int Bc;           // tau points per chunk
};

size_t fixed_bytes(const AdjGeom &g) {
  const int N = g.N;
  size_t b = aligned_bytes((size_t)N * g.nn, 8) + rsplit_bytes(1, N, N) + rsplit_bytes(1, (int)g.nn, N);
  b += aligned_bytes((size_t)N * g.nnp, 4);                                       // Um
  b += 2 * aligned_bytes((size_t)g.NR * g.Kp * g.Kp, 2);                          // U1 split
  b += 2 * aligned_bytes((size_t)g.n * g.NR * g.Kp, 2);                           // U2 split
  b += aligned_bytes((size_t)N * g.n * g.np4, 4) + aligned_bytes((size_t)g.n * N * g.np4, 4);   // U1bar, U2bar
  b += aligned_bytes((size_t)g.Nn, 8) + rsplit_bytes(1, N, g.n) + 2 * aligned_bytes((size_t)N * g.np8, 2);   // Xbar, X
  b += aligned_bytes(sizeof(AdjScalars), 4) + 2 * aligned_bytes(8192, 4) + (1 << 16);
  b += 2 * aligned_bytes((size_t)g.T * g.Nn, 8) + aligned_bytes((size_t)g.T, 4);   // G_Rq, G_wP^T of every tau
  b += aligned_bytes((size_t)N * g.np4, 4);                                        // Xbar of one chunk (FP32)
  return b;
}

size_t per_tau_bytes(const AdjGeom &g) {
  const int n = g.n, N = g.N;
  size_t b = rsplit_bytes(1, N, n) + 2 * aligned_bytes((size_t)N * g.ldN, 4);           // M1 split, E, Ebar
  b += 4 * aligned_bytes((size_t)g.NR * g.Kp, 2);                                 // GR~, GWt~
  b += 2 * aligned_bytes((size_t)g.RG * g.Kp, 2) + 2 * aligned_bytes((size_t)n * g.Kp, 2);   // G(-tau) splits
  b += 2 * aligned_bytes((size_t)n * g.NR * g.Kp, 2);                             // A~
  b += 4 * aligned_bytes((size_t)n * g.Rp * g.Rp, 2);                             // Bbar, Cbar pairs [v][R][P]
  b += aligned_bytes((size_t)n * N * g.np4, 4) + 2 * aligned_bytes((size_t)n * g.abar_pitch, 2);   // Abar, split
  b += 2 * aligned_bytes((size_t)N * g.np4, 4);                                   // GRbar, GWtbar
  b += 2 * aligned_bytes((size_t)N * g.ldN8, 2) + 2 * aligned_bytes((size_t)N * g.np4, 4);   // Ebar pairs, m1, m2
  b += 2 * aligned_bytes((size_t)4 * N * g.np8, 2) + 2 * aligned_bytes((size_t)4 * n * g.np8, 2);   // Xbar operands
  b += 3 * 4096;                                                                  // os, cg, em
  return b;
}

size_t end_bytes(const AdjGeom &g) {
  const int N = g.N;
  return aligned_bytes((size_t)N * g.nnp, 4) + 2 * rsplit_bytes(1, N, (int)g.nn) + rsplit_bytes(1, N, N) +
         rsplit_bytes(1, (int)g.nn, N) + aligned_bytes((size_t)N * g.ldN, 4) + aligned_bytes((size_t)N * g.nnp, 4);
}

AdjGeom adj_geom(sox_handle h, int n, int N, int T, int S) {
  AdjGeom g{};
  g.n = n; g.N = N; g.T = T; g.S = S;
  g.Kp = rup(n, 64);
  g.NR = std::max(N, 128);
  g.RG = std::max(g.Kp, 128);
  g.Rp = rup(N, 128);
  g.nn = (long long)n * n;
  g.np4 = rup4(n);
  g.np8 = (n + 7) & ~7LL;
  g.nnp = rup4(g.nn);
  g.ldN = rup4(N);
  g.ldN8 = (N + 7) & ~7LL;   // FP16 rows: a TMA row stride is a multiple of 16 bytes
  g.Nn = (long long)N * n;
  g.abar_pitch = (g.Nn + 7) & ~7LL;
  const size_t per = per_tau_bytes(g);
  // 64 GB by default: the largest batch instances (about 9 GB per tau at n = 298) then take
  // several tau points per chunk, so the per-chunk launches fill whole waves of the SMs (one
  // tau point of n = 298 is 196 fused-producer tiles, 1.3 waves on 152 SMs)
  const size_t budget = chunk_budget(h, size_t(64) << 30);
  long long c = (long long)(budget / std::max<size_t>(per, 1));
  c = std::max<long long>(1, std::min<long long>({c, (long long)T, 1024}));
  g.Bc = (int)c;
  return g;
}

}  // namespace

size_t adjoint_tc_bytes(sox_handle h, int n, int N, int T, int S) {
  const AdjGeom g = adj_geom(h, n, N, T, S);
  return fixed_bytes(g) + std::max(per_tau_bytes(g) * g.Bc, end_bytes(g)) + (1 << 20);
}

Status phi_adjoint_xv_tc(sox_handle h, int n, int N, int T, int S, const double *G, const double *X, const double *V,
                         const double *w, const double *dphi, double *dX, double *dV, Arena &ar, cudaStream_t s) {
  const AdjGeom g = adj_geom(h, n, N, T, S);
  const long long nn = g.nn, Nn = g.Nn, NN = (long long)N * N;
  const int Kp = g.Kp, NR = g.NR, RG = g.RG, Bc = g.Bc;
  std::string err;
  // ---- set-up: mixed tensor in FP32 and its per-tensor splits; accumulators
  double *Y = ar.take<double>((size_t)N * nn);
  CSplit Vs = rsplit_take(ar, 1, N, N), Ys = rsplit_take(ar, 1, (int)nn, N);
  float *Um = ar.take<float>((size_t)N * g.nnp);
  __half *U1h = ar.take<__half>((size_t)NR * Kp * Kp), *U1l = ar.take<__half>((size_t)NR * Kp * Kp);
  __half *U2h = ar.take<__half>((size_t)n * NR * Kp), *U2l = ar.take<__half>((size_t)n * NR * Kp);
  float *U1bar = ar.take<float>((size_t)N * n * g.np4), *U2bar = ar.take<float>((size_t)n * N * g.np4);
  double *Xbar = ar.take<double>((size_t)Nn);
  CSplit Xr = rsplit_take(ar, 1, N, n);   // X rows R, K = t (E = M1 X^T)
  __half *Xh = ar.take<__half>((size_t)N * g.np8), *Xl = ar.take<__half>((size_t)N * g.np8);   // X pairs [R][t]
  AdjScalars *sc = ar.take<AdjScalars>(1);
  float *cgb = ar.take<float>(2048), *emb = ar.take<float>(2048);
  double *GRall = ar.take<double>((size_t)T * Nn), *GWall = ar.take<double>((size_t)T * Nn);   // one spin
  int *symf = ar.take<int>((size_t)T);
  float *Xbf = ar.take<float>((size_t)N * g.np4);
  if (!Xbf) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  ProfScope ps(h, "phi_adjoint_tc", s, 0);
  long long launches = 0;
  SOX_CUDA_TRY(cudaMemsetAsync(U1bar, 0, 4 * (size_t)N * n * g.np4, s));
  SOX_CUDA_TRY(cudaMemsetAsync(U2bar, 0, 4 * (size_t)n * N * g.np4, s));
  SOX_CUDA_TRY(cudaMemsetAsync(Xbar, 0, 8 * (size_t)Nn, s));
  SOX_CUDA_TRY(cudaMemsetAsync(U1h, 0, 2 * (size_t)NR * Kp * Kp, s));
  SOX_CUDA_TRY(cudaMemsetAsync(U1l, 0, 2 * (size_t)NR * Kp * Kp, s));
  SOX_CUDA_TRY(cudaMemsetAsync(U2h, 0, 2 * (size_t)n * NR * Kp, s));
  SOX_CUDA_TRY(cudaMemsetAsync(U2l, 0, 2 * (size_t)n * NR * Kp, s));
  SOX_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(AdjScalars), s));
  launch_pair_products_f64(X, Y, N, n, s);
  rsplit(V, false, 0, N, 0, 0, 1, 1, N, N, Vs, s);
  rsplit(Y, false, 0, 1, 0, 0, nn, 1, (int)nn, N, Ys, s);                  // rows (a,b), K = Q
  SOX_TRY(cgemm_tc(h, Vs, Ys, 1, nullptr, nullptr, 1.f, Um, g.nnp, 0, s));   // Um[P][(a,b)]
  // one scale for the mixed tensor in both slots: U1 rows (P, q), K = s; U2 [v][R][w]
  launch_absmax(Um, true, g.nnp, N, 0, 1, 1, (int)nn, &sc->mx[2], s);
  launch_split_tensor(Um, true, n, n, g.nnp, N, 1, n, Kp, (long long)Kp * Kp, 1.f, &sc->mx[2], nullptr, U1h, U1l,
                      &sc->sc[kScU], s);
  launch_split_tensor(Um, true, g.nnp, N, n, n, 1, n, Kp, (long long)NR * Kp, 1.f, nullptr, &sc->sc[kScU], U2h, U2l,
                      nullptr, s);
  rsplit(X, false, 0, n, 0, 0, 1, 1, N, n, Xr, s);
  launch_absmax(X, false, n, N, 0, 1, 1, n, &sc->mx[3], s);
  launch_split_tensor(X, false, n, N, 0, 1, 1, n, g.np8, 0, 1.f, &sc->mx[3], nullptr, Xh, Xl, &sc->sc[kScX], s);
  launches += 10;

  // ---- per tau-chunk buffers
  Arena at = ar;
  const size_t Bs = (size_t)Bc;
  CSplit M1s = rsplit_take(at, Bc, N, n);
  float *E = at.take<float>(Bs * N * g.ldN), *Ebar = at.take<float>(Bs * N * g.ldN);
  __half *GRh = at.take<__half>(Bs * NR * Kp), *GRl = at.take<__half>(Bs * NR * Kp);
  __half *GWh = at.take<__half>(Bs * NR * Kp), *GWl = at.take<__half>(Bs * NR * Kp);
  __half *GmTh = at.take<__half>(Bs * RG * Kp), *GmTl = at.take<__half>(Bs * RG * Kp);   // rows v, K = s
  __half *Gmh = at.take<__half>(Bs * n * Kp), *Gml = at.take<__half>(Bs * n * Kp);       // rows s, K = v
  __half *Ah = at.take<__half>(Bs * n * NR * Kp), *Al = at.take<__half>(Bs * n * NR * Kp);
  __half *Bbh = at.take<__half>(Bs * n * g.Rp * g.Rp), *Bbl = at.take<__half>(Bs * n * g.Rp * g.Rp);
  __half *Cbh = at.take<__half>(Bs * n * g.Rp * g.Rp), *Cbl = at.take<__half>(Bs * n * g.Rp * g.Rp);
  float *Abar = at.take<float>(Bs * n * N * g.np4);
  __half *Abh = at.take<__half>(Bs * n * g.abar_pitch), *Abl = at.take<__half>(Bs * n * g.abar_pitch);
  float *GRbf = at.take<float>(Bs * N * g.np4), *GWbf = at.take<float>(Bs * N * g.np4);
  __half *Ebh = at.take<__half>(Bs * N * g.ldN8), *Ebl = at.take<__half>(Bs * N * g.ldN8);   // Ebar pairs
  float *m1f = at.take<float>(Bs * N * g.np4), *m2f = at.take<float>(Bs * N * g.np4);
  // Xbar GEMM operands: A [b][t][R][k] = GRbar, GWtbar, m1, m2; B [b][t][p][k] = G(tau_b)[p][k],
  // G(tau_b)[k][p], -G(-tau_b)[p][k], -G(-tau_b)[k][p]  (K = (b, t, k))
  __half *Xah = at.take<__half>(Bs * 4 * N * g.np8), *Xal = at.take<__half>(Bs * 4 * N * g.np8);
  __half *Xbh = at.take<__half>(Bs * 4 * n * g.np8), *Xbl = at.take<__half>(Bs * 4 * n * g.np8);
  float *osv = at.take<float>(1024);
  if (!osv) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  // zero padding rows and columns that the splits do not write (rows R >= N of GR~ / GWt~,
  // rows v >= n of G(-tau)^T); the splits rewrite every valid element each chunk
  SOX_CUDA_TRY(cudaMemsetAsync(GRh, 0, 2 * Bs * NR * Kp, s));
  SOX_CUDA_TRY(cudaMemsetAsync(GRl, 0, 2 * Bs * NR * Kp, s));
  SOX_CUDA_TRY(cudaMemsetAsync(GWh, 0, 2 * Bs * NR * Kp, s));
  SOX_CUDA_TRY(cudaMemsetAsync(GWl, 0, 2 * Bs * NR * Kp, s));
  SOX_CUDA_TRY(cudaMemsetAsync(GmTh, 0, 2 * Bs * RG * Kp, s));
  SOX_CUDA_TRY(cudaMemsetAsync(GmTl, 0, 2 * Bs * RG * Kp, s));
  SOX_CUDA_TRY(cudaMemsetAsync(E, 0, 4 * Bs * N * g.ldN, s));      // pad columns stay zero
  SOX_CUDA_TRY(cudaMemsetAsync(Ebar, 0, 4 * Bs * N * g.ldN, s));
  // A-GEMM output scale: |A~| <= n 2^15 2^15 os <= 2^15
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  const float os = ldexpf(1.f, -15 - lg);
  k_fill<<<(Bc + 255) / 256, 256, 0, s>>>(osv, Bc, os);
  launches += 1;

  // ---- tensor maps of the fixed-address per-chunk buffers
  CUtensorMap agemm[6], prod[8];
  if (!make_tmap_f16_3d(&agemm[0], GmTh, Kp, RG, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&agemm[1], GmTl, Kp, RG, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&agemm[2], U1h, Kp, (uint64_t)NR * Kp, 1, 64, 128, &err) ||
      !make_tmap_f16_3d(&agemm[3], U1l, Kp, (uint64_t)NR * Kp, 1, 64, 128, &err) ||
      !make_tmap_f16_store4d(&agemm[4], Ah, Kp, NR, n, Bc, &err) ||
      !make_tmap_f16_store4d(&agemm[5], Al, Kp, NR, n, Bc, &err) ||
      !make_tmap_f16_3d(&prod[0], Ah, Kp, NR, (uint64_t)Bc * n, 64, 128, &err) ||
      !make_tmap_f16_3d(&prod[1], Al, Kp, NR, (uint64_t)Bc * n, 64, 128, &err) ||
      !make_tmap_f16_3d(&prod[2], GRh, Kp, NR, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&prod[3], GRl, Kp, NR, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&prod[4], GWh, Kp, NR, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&prod[5], GWl, Kp, NR, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&prod[6], U2h, Kp, NR, n, 64, 128, &err) ||
      !make_tmap_f16_3d(&prod[7], U2l, Kp, NR, n, 64, 128, &err))
    return {SOX_ERR_CUDA, "adjoint maps: " + err};
  // the handle's v range (sox_set_v_range): Phi's v sum, and with it every reverse
  // contraction over v, runs over [v_lo, v_hi); Bbar / Cbar / Abar hold the nv local slices
  int v_lo = 0, v_hi = n;
  v_range(h, n, &v_lo, &v_hi);
  const int nv = v_hi - v_lo;
  const int Kpv = rup(std::max(nv, 1), 64);
  const uint64_t zBC = (uint64_t)Bc * std::max(nv, 1);   // (tau, local v) slices of Bbar / Cbar
  // (i) Abar[b][v][P][q] = sum_R Bbar[b][v][R][P] GR~[b][R][q]: A MN-major, B MN-major
  CUtensorMap mi[5], mii[5], miii[5], miv[5], mv[5], mm1[5], mm2[5], mxb[5];
  const uint64_t sPR = (uint64_t)g.Rp * g.Rp;   // one (tau, v) slice of the pairs: rows R, P contiguous
  if (!make_tmap_f16_3d_rs(&mi[0], Bbh, N, g.Rp, N, zBC, sPR, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&mi[1], Bbl, N, g.Rp, N, zBC, sPR, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&mi[2], GRh, n, Kp, N, Bc, (uint64_t)NR * Kp, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&mi[3], GRl, n, Kp, N, Bc, (uint64_t)NR * Kp, 64, 64, &err) ||
      !make_tmap_f32_store3d(&mi[4], Abar, n, N, zBC, g.np4, (uint64_t)N * g.np4, &err) ||
      // (ii) GRbar[b][R][q] = sum_{v,P} Bbar[b][v][R][P] A~[b][v][P][q]: A K-major, B MN-major
      !make_tmap_f16_3d_rs(&mii[0], Bbh, N, g.Rp, N, zBC, sPR, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mii[1], Bbl, N, g.Rp, N, zBC, sPR, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mii[2], Ah, n, Kp, N, (uint64_t)Bc * n, (uint64_t)NR * Kp, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&mii[3], Al, n, Kp, N, (uint64_t)Bc * n, (uint64_t)NR * Kp, 64, 64, &err) ||
      !make_tmap_f32_store3d(&mii[4], GRbf, n, N, Bc, g.np4, (uint64_t)N * g.np4, &err) ||
      // (iii) GWtbar[b][P][w] = sum_{v,R} Cbar[b][v][R][P] U2~[v][R][w]: A MN-major, B MN-major
      !make_tmap_f16_3d_rs(&miii[0], Cbh, N, g.Rp, N, zBC, sPR, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&miii[1], Cbl, N, g.Rp, N, zBC, sPR, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&miii[2], U2h, n, Kp, N, n, (uint64_t)NR * Kp, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&miii[3], U2l, n, Kp, N, n, (uint64_t)NR * Kp, 64, 64, &err) ||
      !make_tmap_f32_store3d(&miii[4], GWbf, n, N, Bc, g.np4, (uint64_t)N * g.np4, &err) ||
      // (iv) U2bar[v][R][w] += sum_{b,P} Cbar[b][v][R][P] GWt~[b][P][w]: A K-major, B MN-major
      !make_tmap_f16_3d_rs(&miv[0], Cbh, N, g.Rp, N, zBC, sPR, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&miv[1], Cbl, N, g.Rp, N, zBC, sPR, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&miv[2], GWh, n, Kp, N, Bc, (uint64_t)NR * Kp, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&miv[3], GWl, n, Kp, N, Bc, (uint64_t)NR * Kp, 64, 64, &err) ||
      !make_tmap_f32_store3d(&miv[4], U2bar + (size_t)v_lo * N * g.np4, n, N, std::max(nv, 1), g.np4,
                             (uint64_t)N * g.np4, &err) ||
      // (v) U1bar[(P,q)][s] += sum_{b,v} Abar~[b][v][(P,q)] G(-tau_b)~[s][v]: A MN-major, B K-major
      !make_tmap_f16_3d_rs(&mv[0], Abh, Nn, g.abar_pitch, std::max(nv, 1), Bc,
                           (uint64_t)std::max(nv, 1) * g.abar_pitch, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&mv[1], Abl, Nn, g.abar_pitch, std::max(nv, 1), Bc,
                           (uint64_t)std::max(nv, 1) * g.abar_pitch, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&mv[2], Gmh, std::max(nv, 1), Kpv, n, Bc, (uint64_t)n * Kpv, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mv[3], Gml, std::max(nv, 1), Kpv, n, Bc, (uint64_t)n * Kpv, 64, 128, &err) ||
      !make_tmap_f32_store3d(&mv[4], U1bar, n, Nn, 1, g.np4, (uint64_t)Nn * g.np4, &err) ||
      // m1[b][P][t] = sum_R Ebar[b][P][R] X[R][t] (A K-major), m2[b][R][t] = sum_P Ebar[b][P][R] X[P][t]
      // (A MN-major); X pairs [R][t] MN-major in both
      !make_tmap_f16_3d_rs(&mm1[0], Ebh, N, g.ldN8, N, Bc, (uint64_t)N * g.ldN8, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mm1[1], Ebl, N, g.ldN8, N, Bc, (uint64_t)N * g.ldN8, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mm1[2], Xh, n, g.np8, N, 1, (uint64_t)N * g.np8, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&mm1[3], Xl, n, g.np8, N, 1, (uint64_t)N * g.np8, 64, 64, &err) ||
      !make_tmap_f32_store3d(&mm1[4], m1f, n, N, Bc, g.np4, (uint64_t)N * g.np4, &err) ||
      !make_tmap_f16_3d_rs(&mm2[0], Ebh, N, g.ldN8, N, Bc, (uint64_t)N * g.ldN8, 64, 64, &err) ||
      !make_tmap_f16_3d_rs(&mm2[1], Ebl, N, g.ldN8, N, Bc, (uint64_t)N * g.ldN8, 64, 64, &err) ||
      !make_tmap_f32_store3d(&mm2[4], m2f, n, N, Bc, g.np4, (uint64_t)N * g.np4, &err) ||
      // Xbar[R][p] = sum_{b,t,k} A[b][t][R][k] B[b][t][p][k]: both K-major
      !make_tmap_f16_3d_rs(&mxb[0], Xah, n, g.np8, N, 4 * (uint64_t)Bc, (uint64_t)N * g.np8, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mxb[1], Xal, n, g.np8, N, 4 * (uint64_t)Bc, (uint64_t)N * g.np8, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mxb[2], Xbh, n, g.np8, n, 4 * (uint64_t)Bc, (uint64_t)n * g.np8, 64, 128, &err) ||
      !make_tmap_f16_3d_rs(&mxb[3], Xbl, n, g.np8, n, 4 * (uint64_t)Bc, (uint64_t)n * g.np8, 64, 128, &err) ||
      !make_tmap_f32_store3d(&mxb[4], Xbf, n, N, 1, g.np4, (uint64_t)N * g.np4, &err))
    return {SOX_ERR_CUDA, "adjoint maps: " + err};
  mm2[2] = mm1[2];
  mm2[3] = mm1[3];
  const int kcN = (N + 63) / 64;
  const int sms = h->sm_count;
  const long long limit = h->spin_limit;

  for (int sp = 0; sp < S && nv > 0; ++sp) {
    {  // FP64 projections of every tau of this spin: G_Rq = X G(tau), G_wP^T = X G(tau)^T
       // (copied from G_Rq where G(tau) is symmetric); M1 below reuses G_Rq of the mirror point
      const double *Gs = G + (long long)sp * T * nn;
      launch_symmetry_flags(Gs, n, T, symf, s);
      GemmF64 a;
      a.M = N; a.Nc = n; a.K = n; a.batch = T;
      a.A = X; a.ai = n; a.ak = 1;
      a.B = Gs; a.sB = nn; a.bk = n; a.bj = 1;
      a.C = GRall; a.sC = Nn; a.ci = n; a.cj = 1;
      launch_gemm_f64(a, s);
      GemmF64 b = a;
      b.bk = 1; b.bj = n; b.C = GWall; b.skip = symf;
      launch_gemm_f64(b, s);
      k_copy_flagged<<<grid1((long long)T * Nn), 256, 0, s>>>(GRall, GWall, Nn, T, symf);
      launches += 4;
    }
    for (int j0 = 0; j0 < T; j0 += Bc) {
      const int bc = std::min(Bc, T - j0);
      const double *Gj = G + ((long long)sp * T + j0) * nn;                 // G(tau_j), b = 0..bc-1
      const double *Gm0 = G + ((long long)sp * T + (T - 1 - j0)) * nn;      // G(tau_{T-1-j}); stride -nn
      const double *GR = GRall + (long long)j0 * Nn, *GWt = GWall + (long long)j0 * Nn;
      // E = X G(-tau) X^T = -(X G(tau_{T-1-j})) X^T: G_Rq of the mirror points (batch stride -Nn)
      rsplit(GRall + (long long)(T - 1 - j0) * Nn, false, -Nn, n, 0, 0, 1, bc, N, n, M1s, s);
      SOX_TRY(cgemm_tc(h, M1s, Xr, bc, nullptr, nullptr, -1.f, E, g.ldN, (long long)N * g.ldN, s));
      // per-chunk maxima and scales
      SOX_CUDA_TRY(cudaMemsetAsync(sc->mx, 0, sizeof(sc->mx[0]) * 2, s));       // E, Abar
      SOX_CUDA_TRY(cudaMemsetAsync(&sc->mx[4], 0, sizeof(sc->mx[0]) * 4, s));   // G(-tau), GR, GWt, Ebar
      float *mxGR = &sc->mx[5], *mxGW = &sc->mx[6], *mxGm = &sc->mx[4];
      launch_absmax(E, true, g.ldN, N, (long long)N * g.ldN, bc, 1, N, &sc->mx[0], s);
      launch_absmax(GR, false, n, N, Nn, bc, 1, n, mxGR, s);
      launch_absmax(GWt, false, n, N, Nn, bc, 1, n, mxGW, s);
      launch_absmax(Gm0, false, n, n, -nn, bc, 1, n, mxGm, s);
      launch_split_tensor(GR, false, n, N, Nn, bc, 1, n, Kp, (long long)NR * Kp, 1.f, mxGR, nullptr, GRh, GRl,
                          &sc->sc[kScGR], s);
      launch_split_tensor(GWt, false, n, N, Nn, bc, 1, n, Kp, (long long)NR * Kp, 1.f, mxGW, nullptr, GWh, GWl,
                          &sc->sc[kScGW], s);
      // G(-tau_b) = -G(tau_{T-1-j}): transposed (rows v, K = s) for the A-GEMM, and rows s, K = v
      launch_split_tensor(Gm0, false, 1, n, -nn, bc, n, n, Kp, (long long)RG * Kp, -1.f, mxGm, nullptr, GmTh, GmTl,
                          &sc->sc[kScGm], s);
      launch_split_tensor(Gm0 + v_lo, false, n, n, -nn, bc, 1, nv, Kpv, (long long)n * Kpv, -1.f, mxGm, nullptr,
                          Gmh, Gml, nullptr, s);   // columns v in the range only
      k_adj_factors<<<1, 256, 0, s>>>(sc, w, dphi + sp, j0, bc, n, os, cgb, emb);
      launches += 14;
      {  // A~[b][v][P][q] = os sum_s G(-tau_b)~[s][v] U1~[(P,q)][s]
        GemmTcArgs ga;
        ga.M = n; ga.Ncols = NR * Kp; ga.Kp = Kp; ga.K = n; ga.batch = bc;
        ga.batchA_shared = 0; ga.batchB_shared = 1;
        ga.mode = kStoreSplit;
        ga.out_scale = osv;
        ga.group = Kp; ga.n_groups = NR;
        ga.spin_limit = limit; ga.status = h->d_status;
        const long long tiles = (long long)bc * ((n + 127) / 128) * (((long long)NR * Kp + 127) / 128);
        SOX_CUDA_TRY(launch_gemm_f16x2(agemm, ga, (int)std::max<long long>(1, std::min<long long>(tiles, sms)), s));
      }
      {  // fused producer: Bbar, Cbar pairs and Ebar
        AdjBcArgs pa;
        pa.n = n; pa.N = N; pa.Kp = Kp; pa.batch = bc;
        pa.v0 = v_lo; pa.v1 = v_hi;
        pa.spin_limit = limit; pa.status = h->d_status;
        pa.E = E; pa.ldE = g.ldN; pa.sE = (long long)N * g.ldN;
        pa.cg = cgb; pa.em = emb;
        pa.Ebar = Ebar;
        pa.Bh = Bbh; pa.Bl = Bbl; pa.Ch = Cbh; pa.Cl = Cbl; pa.Rp = g.Rp;
        const long long tiles = (long long)bc * ((N + 127) / 128) * ((N + 127) / 128);
        ProfScope pp(h, "adj_bc", s);
        SOX_CUDA_TRY(launch_adj_bc(prod, pa, (int)std::max<long long>(1, std::min<long long>(tiles, sms)), s));
      }
      launches += 2;
      {
        ProfScope pg(h, "adj_gemm", s, 4);
        // (i) Abar (per (b, v); K = R)
        GemmMnArgs a1;
        a1.M = N; a1.Ncols = n; a1.batch = bc * nv; a1.kc_inner = kcN; a1.nk_outer = 1;
        a1.a.mn_major = 1; a1.a.zb = 1;   // pairs [R][P]: rows P run along the MN side
        a1.b.mn_major = 1; a1.b.zb = 1; a1.b.zdiv = nv;
        a1.alpha = &sc->f[kFacAbar];
        a1.spin_limit = limit; a1.status = h->d_status;
        SOX_CUDA_TRY(launch_gemm_mn(mi, a1, plan_gemm_mn(a1, sms, 1), s));
        // (ii) GRbar (per b; K = (v, P))
        SOX_CUDA_TRY(cudaMemsetAsync(GRbf, 0, 4 * (size_t)bc * N * g.np4, s));
        GemmMnArgs a2;
        a2.M = N; a2.Ncols = n; a2.batch = bc; a2.kc_inner = kcN; a2.nk_outer = nv;
        a2.a.mn_major = 0; a2.a.zb = nv; a2.a.zk = 1;
        a2.b.mn_major = 1; a2.b.zb = n; a2.b.zk = 1; a2.b.z0 = v_lo;
        a2.alpha = &sc->f[kFacGRbar];
        a2.spin_limit = limit; a2.status = h->d_status;
        SOX_CUDA_TRY(launch_gemm_mn(mii, a2, plan_gemm_mn(a2, sms, 64), s));
        // (iii) GWtbar (per b; K = (v, R))
        SOX_CUDA_TRY(cudaMemsetAsync(GWbf, 0, 4 * (size_t)bc * N * g.np4, s));
        GemmMnArgs a3;
        a3.M = N; a3.Ncols = n; a3.batch = bc; a3.kc_inner = kcN; a3.nk_outer = nv;
        a3.a.mn_major = 1; a3.a.zb = nv; a3.a.zk = 1;
        a3.b.mn_major = 1; a3.b.zb = 0; a3.b.zk = 1; a3.b.z0 = v_lo;
        a3.alpha = &sc->f[kFacGWtbar];
        a3.spin_limit = limit; a3.status = h->d_status;
        SOX_CUDA_TRY(launch_gemm_mn(miii, a3, plan_gemm_mn(a3, sms, 64), s));
        // (iv) U2bar (per v; K = (b, P)), accumulated over tau
        GemmMnArgs a4;
        a4.M = N; a4.Ncols = n; a4.batch = nv; a4.kc_inner = kcN; a4.nk_outer = bc;
        a4.a.mn_major = 0; a4.a.zb = 1; a4.a.zk = nv;
        a4.b.mn_major = 1; a4.b.zb = 0; a4.b.zk = 1;
        a4.alpha = &sc->f[kFacU2bar];
        a4.accumulate = 1;
        a4.spin_limit = limit; a4.status = h->d_status;
        SOX_CUDA_TRY(launch_gemm_mn(miv, a4, plan_gemm_mn(a4, sms, 64), s));
      }
      // (v) U1bar += Abar (x) G(-tau): Abar split once per chunk, then K = (b, v)
      launch_absmax(Abar, true, g.np4, N, (long long)N * g.np4, bc * nv, 1, n, &sc->mx[1], s);
      launch_split_tensor(Abar, true, g.np4, N, (long long)N * g.np4, bc * nv, 1, n, n, g.abar_pitch, 1.f, &sc->mx[1],
                          nullptr, Abh, Abl, &sc->sc[kScAbar], s);
      k_u1bar_factor<<<1, 1, 0, s>>>(sc);
      {
        GemmMnArgs a5;
        a5.M = (int)Nn; a5.Ncols = n; a5.batch = 1; a5.kc_inner = (nv + 63) / 64; a5.nk_outer = bc;
        a5.a.mn_major = 1; a5.a.zb = 0; a5.a.zk = 1;
        a5.b.mn_major = 0; a5.b.zb = 0; a5.b.zk = 1;
        a5.alpha = &sc->f[kFacU1bar];
        a5.accumulate = 1;
        a5.spin_limit = limit; a5.status = h->d_status;
        SOX_CUDA_TRY(launch_gemm_mn(mv, a5, plan_gemm_mn(a5, sms, 1), s));
      }
      launches += 11;
      // ---- Xbar += sum_b GRbar_b G(tau_b)^T + GWtbar_b G(tau_b) - m1_b G(-tau_b)^T - m2_b G(-tau_b)
      // (m1 = Ebar X, m2 = Ebar^T X; G(-tau_b) = -G(tau_{T-1-j}) enters through the signs): one
      // split GEMM over K = (b, term, k), its FP32 result added to the FP64 accumulator
      launch_absmax(Ebar, true, g.ldN, N, (long long)N * g.ldN, bc, 1, N, &sc->mx[7], s);
      launch_split_tensor(Ebar, true, g.ldN, N, (long long)N * g.ldN, bc, 1, N, g.ldN8, (long long)N * g.ldN8, 1.f,
                          &sc->mx[7], nullptr, Ebh, Ebl, &sc->sc[kScEbar], s);
      k_ex_factor<<<1, 1, 0, s>>>(sc);
      {
        GemmMnArgs e1;
        e1.M = N; e1.Ncols = n; e1.batch = bc; e1.kc_inner = kcN; e1.nk_outer = 1;
        e1.a.mn_major = 0; e1.a.zb = 1;
        e1.b.mn_major = 1;
        e1.alpha = &sc->f[kFacEX];
        e1.spin_limit = limit; e1.status = h->d_status;
        SOX_CUDA_TRY(launch_gemm_mn(mm1, e1, plan_gemm_mn(e1, sms, 1), s));
        GemmMnArgs e2 = e1;
        e2.a.mn_major = 1;
        SOX_CUDA_TRY(launch_gemm_mn(mm2, e2, plan_gemm_mn(e2, sms, 1), s));
      }
      SOX_CUDA_TRY(cudaMemsetAsync(&sc->mx[kMxXa], 0, 2 * sizeof(float), s));
      const float *xa[4] = {GRbf, GWbf, m1f, m2f};
      for (int t = 0; t < 4; ++t)
        launch_absmax(xa[t], true, g.np4, N, (long long)N * g.np4, bc, 1, n, &sc->mx[kMxXa], s);
      for (int t = 0; t < 4; ++t)
        launch_split_tensor(xa[t], true, g.np4, N, (long long)N * g.np4, bc, 1, n, g.np8, 4LL * N * g.np8, 1.f,
                            &sc->mx[kMxXa], nullptr, Xah + (size_t)t * N * g.np8, Xal + (size_t)t * N * g.np8,
                            t == 0 ? &sc->sc[kScXa] : nullptr, s);
      launch_absmax(Gj, false, n, n, nn, bc, 1, n, &sc->mx[kMxXb], s);
      launch_absmax(Gm0, false, n, n, -nn, bc, 1, n, &sc->mx[kMxXb], s);
      struct XbTerm {
        const double *src;
        long long ld0, ldc, ld1;
        float sign;
      };
      const XbTerm xb[4] = {{Gj, n, 1, nn, 1.f}, {Gj, 1, n, nn, 1.f}, {Gm0, n, 1, -nn, -1.f}, {Gm0, 1, n, -nn, -1.f}};
      for (int t = 0; t < 4; ++t)
        launch_split_tensor(xb[t].src, false, xb[t].ld0, n, xb[t].ld1, bc, xb[t].ldc, n, g.np8, 4LL * n * g.np8,
                            xb[t].sign, &sc->mx[kMxXb], nullptr, Xbh + (size_t)t * n * g.np8,
                            Xbl + (size_t)t * n * g.np8, t == 0 ? &sc->sc[kScXb] : nullptr, s);
      k_xbar_factor<<<1, 1, 0, s>>>(sc);
      SOX_CUDA_TRY(cudaMemsetAsync(Xbf, 0, 4 * (size_t)N * g.np4, s));
      {
        GemmMnArgs x;
        x.M = N; x.Ncols = n; x.batch = 1; x.kc_inner = (n + 63) / 64; x.nk_outer = 4 * bc;
        x.a.mn_major = 0; x.a.zk = 1;
        x.b.mn_major = 0; x.b.zk = 1;
        x.alpha = &sc->f[kFacXbar];
        x.spin_limit = limit; x.status = h->d_status;
        SOX_CUDA_TRY(launch_gemm_mn(mxb, x, plan_gemm_mn(x, sms, 64), s));
      }
      k_add_f64<<<grid1(Nn), 256, 0, s>>>(Xbf, g.np4, N, n, Xbar);
      launches += 22;
    }
  }

  // ---- end: Ubar = U1bar + U2bar; Vbar = Ubar Y^T; Z = V^T Ubar; Xbar += pair adjoint of Z
  Arena ae = ar;   // the per-chunk buffers are free again
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
