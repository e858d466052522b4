// Split-precision GEMM with FP32 output whose operands may sit in shared memory
// K-major or MN-major (gemm_mn.cu), and per-tensor split helpers.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <string>

namespace sox {

// One operand (A or B) of k_gemm_mn, an FP16 pair tensor (hi, lo) read through a 3-D
// TMA map (hi and lo maps alike):
//   mn_major = 0: map dims (K, rows, z), box 64 x 128: each 64-wide K chunk of 128 rows.
//   mn_major = 1: map dims (rows, K, z), box 64 x 64: two boxes per chunk (rows 0-63,
//                 64-127 of the tile), K running down the map's second dimension.
// The map's z coordinate for output batch b and outer K index kz is
// z0 + (b / zdiv) * zb + kz * zk.
struct MnOperand {
  int mn_major = 0;
  long long zb = 0, zk = 0;
  int zdiv = 1;   // the batch term uses b / zdiv
  long long z0 = 0;   // constant offset of the z coordinate
};

// C[b](i, j) (+)= alpha * sum_k A(i, k) B(j, k) with k = (kz, kk), kz < nk_outer,
// kk < 64 * kc_inner (the K chunks of one outer index).  Three FP16 MMAs per product
// (hi*lo + lo*hi + hi*hi), FP32 accumulation in TMEM over windows of `window` chunks whose
// results are added in round-to-nearest FP32 in registers (the tensor core truncates each
// accumulation step; short windows keep that bias at ~window * 4 steps * 2^-23).  `ksplit`
// work items share each 128 x 128 output tile, each over a contiguous range of `cps`
// chunks (a multiple of `window`); their results are reduce-added into C by TMA, so C must
// hold zeros (or the values to add to) when ksplit > 1 or accumulate is set.
struct GemmMnArgs {
  int M = 0, Ncols = 0, batch = 1;
  int kc_inner = 1, nk_outer = 1;
  int window = 16;
  int ksplit = 1;
  long long cps = 0;            // chunks per split item (set by plan_gemm_mn)
  MnOperand a, b;
  const float *alpha = nullptr; // optional device scalar multiplying alpha_host
  float alpha_host = 1.f;
  int accumulate = 0;           // reduce-add into C instead of storing
  long long spin_limit = 0;
  int *status = nullptr;
};

// Chooses cps / ksplit so that every work item has chunks and the grid fills `sms` SMs;
// returns the grid size.
int plan_gemm_mn(GemmMnArgs &a, int sms, int max_ksplit);
// maps: A hi, A lo, B hi, B lo, then the FP32 output map (make_tmap_f32_store3d over
// Ncols x M x batch)
cudaError_t launch_gemm_mn(const CUtensorMap *maps, const GemmMnArgs &a, int grid, cudaStream_t s);

// Per-tensor split of a strided source: element (r1, r0, c) at src + r1 * ld1 + r0 * ld0 +
// c * ldc (FP64 or FP32), r1 < rows1, r0 < rows0, c < cols.
// absmax: atomically raises out[0] to max |x| (out must hold 0 or a smaller value first;
// atomicMax on the bit pattern of non-negative floats).
void launch_absmax(const void *src, bool f32, long long ld0, int rows0, long long ld1, int rows1, long long ldc,
                   int cols, float *out, cudaStream_t s);
// split: hi + lo = sign * x * s written at r1 * ldo1 + r0 * ldo + c, with zeros for
// cols <= c < ldo; s = 2^(14 - floor(log2 absmax)) (largest |x * s| in [2^14, 2^15)), or
// *scale_in when given.  scale_out (optional) receives s.
void launch_split_tensor(const void *src, bool f32, long long ld0, int rows0, long long ld1, int rows1, long long ldc,
                         int cols, long long ldo, long long ldo1, float sign, const float *absmax,
                         const float *scale_in, __half *hi, __half *lo, float *scale_out, cudaStream_t s);

}  // namespace sox
