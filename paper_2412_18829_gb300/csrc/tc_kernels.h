// Launch interfaces of the tensor-core kernels (tc_kernels.cu).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <string>

namespace sox {

enum { kStoreSplit = 1, kStoreSplitGroup = 2, kStoreF32 = 3 };

struct BcdArgs {
  // K extent Kp (a multiple of 64): n valid columns, then zeros; the MMAs of the last
  // 64-wide chunk stop after ceil(n / 16) 16-wide steps in total
  int n = 0, N = 0, Kp = 0, batch = 0;
  int v0 = 0, v1 = 0;                // the v sum runs over [v0, v1) (launch_sox_bcd_tc: v1 <= 0 means n)
  long long spin_limit = 0;
  int *status = nullptr;
  const float *row_scale = nullptr;  // [batch][N]
  const float *col_scale = nullptr;  // [batch][N]
  float *Dt = nullptr;               // [batch][N][ldD]
  long long ldD = 0;
};

// One instance's share of a multi-instance fused launch (launch_sox_bcd_multi): its eight
// operand maps (as for launch_sox_bcd_tc, 64 x 128 boxes), its shapes and outputs, and the
// first global work unit (128 x 128 (P, R) tile of one (spin, tau) batch) it owns.
struct BcdJob {
  CUtensorMap maps[8];
  int n = 0, N = 0, Kp = 0, batch = 0, v0 = 0, v1 = 0;
  const float *row_scale = nullptr, *col_scale = nullptr;
  float *Dt = nullptr;
  long long ldD = 0;
  long long unit0 = 0;
};
constexpr int kMaxBcdJobs = 24;   // the table travels as a kernel parameter (< 32 KB)
struct BcdJobs {
  BcdJob job[kMaxBcdJobs];
  int count = 0;
  long long total = 0;        // work units of all jobs
  long long spin_limit = 0;
  int *status = nullptr;
};

// Output of the split GEMM: FP16 pair tensors [batch][M][n_groups][group] written by
// TMA stores (maps 4 and 5 of launch_gemm_f16x2, see make_tmap_f16_store4d).
struct GemmTcArgs {
  int M = 0, Ncols = 0, Kp = 0, batch = 1;
  int K = 0;   // valid K (operand columns >= K are zero; MMAs stop there); 0 = Kp
  int batchA_shared = 0, batchB_shared = 0;
  int mode = kStoreSplit;
  const float *out_scale = nullptr;   // kStoreSplit: one power of two per batch
  // kStoreSplitGroup: columns form groups of `group` (a multiple of 64) whose rows all lie
  // in one tile (M <= 128); each group gets its own power-of-two scale, written to
  // group_scale[b][group index]
  int group = 128, n_groups = 0;
  float *group_scale = nullptr;
  // kStoreF32: Cf[b * sCb + i * ldc + j] = alpha * acc(i, j) * row_scale[zA * rs_b + i] * col_scale[zB * cs_b + j]
  // (either scale may be NULL); rows >= M and columns >= Ncols are not written.  Cf 16-byte
  // aligned, ldc and sCb multiples of 4; the stores go through the FP32 tensor map passed as
  // the first output map (make_tmap_f32_store3d over Ncols x M x batch).
  float *Cf = nullptr;
  long long ldc = 0, sCb = 0;
  float alpha = 1.f;
  int accumulate = 0;   // kStoreF32: add to Cf instead of overwriting
  const float *row_scale = nullptr, *col_scale = nullptr;
  long long rs_b = 0, cs_b = 0;
  // batch coordinate of the A / B operand for output batch b (overrides batch*_shared)
  const int *idxA = nullptr, *idxB = nullptr;
  long long spin_limit = 0;
  int *status = nullptr;
};

bool make_tmap_f16_3d(CUtensorMap *map, const void *base, uint64_t d0, uint64_t d1, uint64_t d2,
                      uint32_t box0, uint32_t box1, std::string *err);
// the same with `batch_stride` elements between consecutive d2 slices (a multiple of 8)
bool make_tmap_f16_3d_bs(CUtensorMap *map, const void *base, uint64_t d0, uint64_t d1, uint64_t d2,
                         uint64_t batch_stride, uint32_t box0, uint32_t box1, std::string *err);
// and with `row_stride` elements between rows (>= d0, a multiple of 8): a window of d0 columns
bool make_tmap_f16_3d_rs(CUtensorMap *map, const void *base, uint64_t d0, uint64_t row_stride, uint64_t d1,
                         uint64_t d2, uint64_t batch_stride, uint32_t box0, uint32_t box1, std::string *err);
size_t tc_smem_bytes();
bool make_tmap_f16_store4d(CUtensorMap *map, const void *base, uint64_t group, uint64_t n_groups, uint64_t rows,
                           uint64_t batch, std::string *err);
// FP32 output [batch][rows][ld] (cols <= ld valid columns) for the kStoreF32 epilogue's TMA
// stores: base 16-byte aligned, ld and batch_stride multiples of 4 elements
bool make_tmap_f32_store3d(CUtensorMap *map, const void *base, uint64_t cols, uint64_t rows, uint64_t batch,
                           uint64_t ld, uint64_t batch_stride, std::string *err);
// Variants of the fused kernel: G_R / G_wP^T resident in shared memory for the whole
// (spin, tau) batch (Kp <= 128 only), streamed with A_v and U2_v, or streamed on CTA
// pairs (cta_group::2; the grid is then the device's pair capacity, `grid` is ignored).
// maps: 0/1 A hi/lo, 2/3 G_Rq hi/lo, 4/5 G_wP^T hi/lo, 6/7 U2 hi/lo (boxes 64 x 128); the
// pair variant reads 8/9 G_Rq hi/lo and 10/11 U2 hi/lo with 64 x 64 boxes instead of 2/3, 6/7.
enum { kBcdResident = 1, kBcdStreamed = 2, kBcdPair = 3 };
cudaError_t launch_sox_bcd_tc(const CUtensorMap *maps, const BcdArgs &a, int grid, cudaStream_t s, int variant);
// One persistent launch of the streamed fused kernel over the tiles of several instances of
// different sizes (jobs.job[j].unit0 ascending; each job's v range already clamped).
cudaError_t launch_sox_bcd_multi(const BcdJobs &jobs, int grid, cudaStream_t s);
// maps: A hi/lo, B hi/lo (3-D loads), C hi/lo (4-D stores)
cudaError_t launch_gemm_f16x2(const CUtensorMap *maps, const GemmTcArgs &a, int grid, cudaStream_t s);
// rows of batch b come from alt_src instead of src when use_alt[b] != 0 (both optional)
void launch_split_rows_f64(const double *src, long long ld, long long bstride, int rows_valid, int rows_out,
                           int L, int Kp, __half *hi, __half *lo, float *inv_scale, int batch, cudaStream_t s,
                           const double *alt_src = nullptr, const int *use_alt = nullptr);
void launch_mixed_f32(const double *V, const double *X, int N, int n, int Kp, float *U, cudaStream_t s);
void launch_split_mixed(const float *U, int N, int NR, int n, int Kp, __half *u1_hi, __half *u1_lo,
                        __half *u2_hi, __half *u2_lo, float *inv_scale, cudaStream_t s);
void launch_prep_gminus(const double *G, int n, int T, int nbatch, int Kp, __half *hi, __half *lo,
                        float *gscale, float *out_scale, int b0, int rows_out, cudaStream_t s);
void launch_bcd_scales(const float *inv_u1, const float *gsc, const float *osc, const float *asc, int NR,
                       const float *inv_gw, const float *inv_gr, const float *inv_u2, int N, int batch,
                       float *row, float *col, cudaStream_t s);

// SIMT back-projection helpers (FP32 / FP64 accumulate), tc_kernels.cu
void launch_backproject_T(const float *Dt, long long ldD, const double *X, int N, int n, int batch, float *T,
                          cudaStream_t s);
// sym (optional, per batch): when set, Sigma[b] is symmetric and only the upper
// block triangle is computed, then mirrored
void launch_backproject_sigma(const double *X, const float *T, int N, int n, int batch, double *Sigma,
                              long long sstride, cudaStream_t s, const int *sym = nullptr);

}  // namespace sox
