// Tensor-core (tcgen05) kernels of the split-precision path and their helpers.
//
// Split format: a row x of real numbers is stored as two FP16 rows (hi, lo)
// with x * s = hi + lo, s a power of two chosen per row (or per group of rows)
// so that max|x * s| lies in [1, 2).  A product of two split operands is
// evaluated by three FP16 MMAs, hi*hi + hi*lo + lo*hi, accumulated in FP32.
#include <cstdio>
#include <string>

#include "tc_common.cuh"
#include "smem_attr.h"
#include "tc_kernels.h"

namespace sox {

using tc::smem_u32;

bool make_tmap_f16_3d(CUtensorMap *map, const void *base, uint64_t d0, uint64_t d1, uint64_t d2,
                      uint32_t box0, uint32_t box1, std::string *err) {
  return make_tmap_f16_3d_bs(map, base, d0, d1, d2, d0 * d1, box0, box1, err);
}

bool make_tmap_f16_3d_bs(CUtensorMap *map, const void *base, uint64_t d0, uint64_t d1, uint64_t d2,
                         uint64_t batch_stride, uint32_t box0, uint32_t box1, std::string *err) {
  return make_tmap_f16_3d_rs(map, base, d0, d0, d1, d2, batch_stride, box0, box1, err);
}

bool make_tmap_f16_3d_rs(CUtensorMap *map, const void *base, uint64_t d0, uint64_t row_stride, uint64_t d1,
                         uint64_t d2, uint64_t batch_stride, uint32_t box0, uint32_t box1, std::string *err) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      if (err) *err = "cuTensorMapEncodeTiled entry point not available";
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {row_stride * 2, batch_stride * 2};
  cuuint32_t box[3] = {box0, box1, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(base), dims, strides, box,
                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r);
    return false;
  }
  return true;
}

namespace {

constexpr int kTile = 128;              // M and N of every MMA tile
constexpr int kChunk = 64;              // K elements per TMA box (128 bytes of FP16)
constexpr int kTileBytes = kTile * kChunk * 2;  // 16 KB
constexpr int kStageBytes = 4 * kTileBytes;     // hi/lo of both operands
constexpr int kStages = 3;
constexpr uint32_t kIdesc = tc::idesc_f16_f32(kTile, kTile);

// full[q][s]: stage s holds a chunk for MMA issuer q.  Each issuer waits only on its own
// set, so the phases it counts on a barrier are exactly the ones it consumes: on a ring
// shared by two issuers, an issuer that skips the other's chunks would otherwise wait on a
// phase two or more ahead of the barrier, where the parity test reads as complete.
struct Barriers {
  uint64_t full[2][kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

// Waits that let copies and MMAs in flight finish before the CTA exits (or frees
// TMEM) keep a floor independent of the caller's cap, so a tiny cap cannot let
// a TMA write land in shared memory the CTA no longer owns.
__device__ __forceinline__ long long wind_down_limit(long long cap) { return cap > (1LL << 20) ? cap : (1LL << 20); }

__device__ __forceinline__ uint8_t *stage_ptr(uint8_t *smem, int s, int t) {
  return smem + (size_t)s * kStageBytes + (size_t)t * kTileBytes;
}

// Issues the 3 x ks MMAs of one 64-wide K chunk (ks 16-wide steps, 1..4: the last chunk
// of a contraction stops at the first all-padding step):
// acc (+)= (ahi + alo)(bhi + blo)^T minus lo*lo.
// The small cross terms go first: the tensor core truncates every accumulation
// step to FP32 (round toward zero), and each step into a large accumulator
// costs up to one ulp, so the large hi*hi steps are kept last and fewest.
template <int KS>
__device__ __forceinline__ void issue_chunk_ks(uint32_t acc, uint8_t *st, bool first, uint32_t idesc) {
  const uint32_t a_hi = smem_u32(st), a_lo = a_hi + kTileBytes;
  const uint32_t b_hi = a_hi + 2 * kTileBytes, b_lo = a_hi + 3 * kTileBytes;
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
// one straight-line MMA sequence per step count (a loop with a runtime exit between the
// MMAs slowed the issuing thread down measurably)
__device__ __forceinline__ void issue_chunk(uint32_t acc, uint8_t *st, bool first, int ks,
                                            uint32_t idesc = kIdesc) {
  if (ks >= 4) issue_chunk_ks<4>(acc, st, first, idesc);
  else if (ks == 3) issue_chunk_ks<3>(acc, st, first, idesc);
  else if (ks == 2) issue_chunk_ks<2>(acc, st, first, idesc);
  else issue_chunk_ks<1>(acc, st, first, idesc);
}

// Instruction descriptor of a 128-row tile whose N side holds `cols` valid columns from
// `c0` on: N = the valid width rounded up to 16 (at most 128), so no MMA runs over the
// zero rows past the end of the operand
__device__ __forceinline__ uint32_t idesc_cols(int c0, int cols) {
  const int w = cols - c0 >= kTile ? kTile : ((cols - c0 + 15) & ~15);
  return tc::idesc_f16_f32(kTile, w < 16 ? 16 : w);
}

// 16-wide K steps of chunk kc when the contraction has K valid elements (the rest of the
// padded extent is zero): 4, except in the last chunk.
__device__ __forceinline__ int chunk_steps(int kc, int K) {
  const int rem = K - kc * kChunk;
  return rem >= kChunk ? kChunk / 16 : (rem + 15) / 16;
}

__device__ __forceinline__ void setup_barriers(Barriers *bar, int epi_threads) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&bar->full[0][s], 1);
      tc::mbar_init(&bar->full[1][s], 1);
      tc::mbar_init(&bar->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bar->acc_full[b], 1);
      tc::mbar_init(&bar->acc_empty[b], epi_threads);
    }
    tc::mbar_init(&bar->drain, 2);   // one commit per issuing warp
    bar->abort = 0;
    tc::fence_barrier_init();
  }
}

// Fused kernels: warp 0 TMA, warps 1 and 6 MMA, warps 2..5 epilogue (one per TMEM lane
// quarter, 128 columns each).  Measured: the epilogue is not the limit (a variant that
// skips its TMEM loads runs at the same speed), so it stays at four warps with 255
// registers available.
// Two MMA-issuing warps, warp 1 for the B_v halves and warp 6 for the C_v halves, each into
// its own accumulators (so every accumulator receives its MMAs from one thread, in order).
// An issuing thread stalls at each wait for a stage, and the tensor pipe holds few MMAs
// ahead of it, so one issuer leaves the pipe idle at every wait; with two, one issues while
// the other waits.  The producer alternates B and C chunks in the stage ring (B_v chunk kc
// at ring position 2kc, C_v chunk kc at 2kc + 1 of the v's 2 nk positions), so both issuers
// always have a chunk in flight.  Measured on the mid-size build's fused kernel: one issuer
// 9.4 ms, two issuers over B-then-C halves 7.6 ms, alternating chunks 7.1 ms (n = 298: 39.4 ->
// 32.8 ms); the multi-instance kernel keeps the B-then-C order (see there).  Seven warps
// take the same registers as six (registers are granted per four warps).
constexpr int kBcdThreads = 224;
constexpr int kEpiThreads = 128;

// Epilogue of the fused kernels: D[P, R] += B_v[P, R] * C_v[P, R] over v, in
// registers; B_v at TMEM columns [buf*256, +128), C_v at [buf*256 + 128, +128).
// At the end of a tile D is rescaled and written transposed, Dt[b][R][P].
template <class Bar>
__device__ __forceinline__ void bcd_epilogue(Bar *bar, uint32_t tmem, const BcdArgs &a, int tP,
                                             long long total, volatile int *abort, int warp, int lane) {
  const int tiles_per_b = tP * tP;
  const int q = warp & 3;                 // TMEM lane quarter of this warp
  const int row = q * 32 + lane;          // P offset inside the tile
  long long acc_it = 0;
  for (long long t = blockIdx.x; t < total && !*abort; t += gridDim.x) {
    const int b = (int)(t / tiles_per_b);
    const int r = (int)(t % tiles_per_b);
    const int P0 = (r / tP) * kTile, R0 = (r % tP) * kTile;
    float d[kTile];
#pragma unroll
    for (int j = 0; j < kTile; ++j) d[j] = 0.f;
    bool ok = true;
    for (int v = a.v0; v < a.v1; ++v, ++acc_it) {
      const int buf = (int)(acc_it & 1);
      const uint32_t aph = (uint32_t)((acc_it >> 1) & 1);
      ok = tc::mbar_wait(&bar->acc_full[buf], aph, a.spin_limit, abort, a.status, 8);
      if (!ok) break;
      tc::tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + buf * 256;
#pragma unroll
      for (int c = 0; c < kTile; c += 16) {
        float bv[16], cv[16];
        tc::tmem_ld_32x32b_x16(base + c, bv);
        tc::tmem_ld_32x32b_x16(base + 128 + c, cv);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) d[c + j] = fmaf(bv[j], cv[j], d[c + j]);
      }
      tc::tc_fence_before();
      tc::mbar_arrive(&bar->acc_empty[buf]);
    }
    if (!ok) break;
    const int P = P0 + row;
    if (P < a.N) {
      const float rs = a.row_scale[(long long)b * a.N + P];
      float *out = a.Dt + (long long)b * a.N * a.ldD + P;
#pragma unroll
      for (int j = 0; j < kTile; ++j) {
        const int R = R0 + j;
        if (R < a.N) out[(long long)R * a.ldD] = d[j] * rs * a.col_scale[(long long)b * a.N + R];
      }
    }
  }
}

// ============================================================================
// Fused B / C / Hadamard-reduce (Sec. II C, the B, C and D steps):
//   D[b][P][R] = sum_v (sum_q A[b][v][P][q] GR[b][R][q]) (sum_w GW[b][P][w] U2[v][R][w])
// One 128 x 128 (P, R) tile per work item; B_v and C_v accumulate in TMEM
// (double-buffered), the Hadamard product accumulates in registers, and only
// D leaves the SM, written transposed and rescaled: Dt[b][R][P].
// ============================================================================
__global__ void __launch_bounds__(kBcdThreads, 1)
    k_sox_bcd_tc(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
                 const __grid_constant__ CUtensorMap tmGR_hi, const __grid_constant__ CUtensorMap tmGR_lo,
                 const __grid_constant__ CUtensorMap tmGW_hi, const __grid_constant__ CUtensorMap tmGW_lo,
                 const __grid_constant__ CUtensorMap tmU_hi, const __grid_constant__ CUtensorMap tmU_lo,
                 BcdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Barriers *bar = reinterpret_cast<Barriers *>(smem + kStages * kStageBytes);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tP = (a.N + kTile - 1) / kTile;
  const int tiles_per_b = tP * tP;
  const long long total = (long long)a.batch * tiles_per_b;
  const int nk = a.Kp / kChunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&bar->full[0][s], 1);
      tc::mbar_init(&bar->full[1][s], 1);
      tc::mbar_init(&bar->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bar->acc_full[b], 2);   // one commit per issuing warp
      tc::mbar_init(&bar->acc_empty[b], kEpiThreads);
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

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      long long it = 0;
      tc::RingPhases ring;
      for (long long t = blockIdx.x; t < total && !*abort; t += gridDim.x) {
        const int b = (int)(t / tiles_per_b);
        const int r = (int)(t % tiles_per_b);
        const int P0 = (r / tP) * kTile, R0 = (r % tP) * kTile;
        for (int v = a.v0; v < a.v1 && !*abort; ++v) {
          for (int p = 0; p < 2 * nk && !*abort; ++p, ++it) {
            int kc, half;
            tc::bc_decode(p, nk, 1, kc, half);
            const int s = (int)(it % kStages);
            const uint32_t ph = (uint32_t)((it / kStages) & 1);
            if (!tc::mbar_wait(&bar->empty[s], ph ^ 1u, a.spin_limit, abort, a.status, 1)) break;
            uint64_t *fb = &bar->full[half][s];   // the half's issuer
            ring.take(half, s);
            tc::mbar_arrive_expect_tx(fb, kStageBytes);
            const int x = kc * kChunk;
            if (half == 0) {
              tc::tma_load_3d(stage_ptr(smem, s, 0), &tmA_hi, fb, x, P0, b * a.n + v);
              tc::tma_load_3d(stage_ptr(smem, s, 1), &tmA_lo, fb, x, P0, b * a.n + v);
              tc::tma_load_3d(stage_ptr(smem, s, 2), &tmGR_hi, fb, x, R0, b);
              tc::tma_load_3d(stage_ptr(smem, s, 3), &tmGR_lo, fb, x, R0, b);
            } else {
              tc::tma_load_3d(stage_ptr(smem, s, 0), &tmGW_hi, fb, x, P0, b);
              tc::tma_load_3d(stage_ptr(smem, s, 1), &tmGW_lo, fb, x, P0, b);
              tc::tma_load_3d(stage_ptr(smem, s, 2), &tmU_hi, fb, x, R0, v);
              tc::tma_load_3d(stage_ptr(smem, s, 3), &tmU_lo, fb, x, R0, v);
            }
          }
        }
      }
      // wind down: every stage issued must have landed before the CTA exits
      tc::ring_wind_down(bar->full, ring, wind_down_limit(a.spin_limit));
    }
  } else if (warp == 1 || warp == 6) {
    // ---------------- MMA issuers: warp 1 the B_v chunks, warp 6 the C_v chunks ----------------
    if (lane == 0) {
      const int my = (warp == 1) ? 0 : 1;
      long long it = 0, acc_it = 0;
      tc::RingPhases ring;   // this issuer's phases on its set, full[my][.]
      bool ok = true;
      for (long long t = blockIdx.x; t < total && ok && !*abort; t += gridDim.x) {
        const uint32_t idesc = idesc_cols((int)((t % tiles_per_b) % tP) * kTile, a.N);   // R side
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
              const int s = (int)((it + tc::bc_pos(kc, my, nk, 1)) % kStages);
              ok = tc::mbar_wait(&bar->full[my][s], ring.take(my, s), a.spin_limit, abort, a.status, 4);
              if (!ok) break;
              tc::tc_fence_after();
              issue_chunk(acc, stage_ptr(smem, s, 0), kc == 0, chunk_steps(kc, a.n), idesc);
              tc::mma_commit(&bar->empty[s]);
            }
          }
          it += 2 * nk;
          if (ok) tc::mma_commit(&bar->acc_full[buf]);
        }
      }
      // all MMAs complete before TMEM is released
      tc::mma_commit(&bar->drain);
      for (long long i = 0; i < wind_down_limit(a.spin_limit) && !tc::mbar_try_wait(&bar->drain, 0); ++i) {
      }
    }
  } else if (warp >= 2 && warp <= 5) {
    bcd_epilogue(bar, tmem, a, tP, total, abort, warp, lane);
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ============================================================================
// The streamed fused kernel over several instances at once (the uneven batch): one
// persistent grid walks the concatenated tiles of every job; each role (TMA producer, MMA
// issuer, epilogue) decodes the job of a tile from the table in the kernel parameters and
// reads that job's maps, shapes and outputs.  Jobs are ordered by cost, largest first, so
// the grid's last wave holds the cheapest tiles.
// ============================================================================
struct MultiTile {
  int j, b, P0, R0;
};

__device__ __forceinline__ MultiTile multi_tile(const BcdJobs &jobs, long long t) {
  int j = 0;
  while (j + 1 < jobs.count && jobs.job[j + 1].unit0 <= t) ++j;
  const BcdJob &J = jobs.job[j];
  const int tP = (J.N + kTile - 1) / kTile;
  const long long local = t - J.unit0;
  const int per_b = tP * tP;
  MultiTile m;
  m.j = j;
  m.b = (int)(local / per_b);
  const int r = (int)(local % per_b);
  m.P0 = (r / tP) * kTile;
  m.R0 = (r % tP) * kTile;
  return m;
}

__global__ void __launch_bounds__(kBcdThreads, 1) k_sox_bcd_multi(const __grid_constant__ BcdJobs jobs) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Barriers *bar = reinterpret_cast<Barriers *>(smem + kStages * kStageBytes);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const long long total = jobs.total;
  const long long limit = jobs.spin_limit;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&bar->full[0][s], 1);
      tc::mbar_init(&bar->full[1][s], 1);
      tc::mbar_init(&bar->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bar->acc_full[b], 2);   // one commit per issuing warp
      tc::mbar_init(&bar->acc_empty[b], kEpiThreads);
    }
    tc::mbar_init(&bar->drain, 2);
    bar->abort = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(&bar->tmem_base, 512);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = bar->tmem_base;
  volatile int *abort = &bar->abort;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      long long it = 0;
      tc::RingPhases ring;
      // B_v's chunks, then C_v's (group g = nk): over the uneven batch's long launches, which
      // run under the power cap, this order measured 3 % faster than alternating single
      // chunks (1.49 vs 1.53 s of fused kernel per batch forward), although alternating wins
      // 20 % in a single instance's launch (n = 298, 16 tau) and the same in this kernel
      // with a batch of one
      for (long long t = blockIdx.x; t < total && !*abort; t += gridDim.x) {
        const MultiTile m = multi_tile(jobs, t);
        const BcdJob &J = jobs.job[m.j];
        const int nk = J.Kp / kChunk;
        for (int v = J.v0; v < J.v1 && !*abort; ++v) {
          for (int p = 0; p < 2 * nk && !*abort; ++p, ++it) {
            int kc, half;
            tc::bc_decode(p, nk, nk, kc, half);
            const int s = (int)(it % kStages);
            const uint32_t ph = (uint32_t)((it / kStages) & 1);
            if (!tc::mbar_wait(&bar->empty[s], ph ^ 1u, limit, abort, jobs.status, 1)) break;
            uint64_t *fb = &bar->full[half][s];
            ring.take(half, s);
            tc::mbar_arrive_expect_tx(fb, kStageBytes);
            const int x = kc * kChunk;
            if (half == 0) {
              tc::tma_load_3d(stage_ptr(smem, s, 0), &J.maps[0], fb, x, m.P0, m.b * J.n + v);
              tc::tma_load_3d(stage_ptr(smem, s, 1), &J.maps[1], fb, x, m.P0, m.b * J.n + v);
              tc::tma_load_3d(stage_ptr(smem, s, 2), &J.maps[2], fb, x, m.R0, m.b);
              tc::tma_load_3d(stage_ptr(smem, s, 3), &J.maps[3], fb, x, m.R0, m.b);
            } else {
              tc::tma_load_3d(stage_ptr(smem, s, 0), &J.maps[4], fb, x, m.P0, m.b);
              tc::tma_load_3d(stage_ptr(smem, s, 1), &J.maps[5], fb, x, m.P0, m.b);
              tc::tma_load_3d(stage_ptr(smem, s, 2), &J.maps[6], fb, x, m.R0, v);
              tc::tma_load_3d(stage_ptr(smem, s, 3), &J.maps[7], fb, x, m.R0, v);
            }
          }
        }
      }
      // wind down: every stage issued must have landed before the CTA exits
      tc::ring_wind_down(bar->full, ring, wind_down_limit(limit));
    }
  } else if (warp == 1 || warp == 6) {
    // ---------------- MMA issuers: warp 1 the B_v chunks, warp 6 the C_v chunks ----------------
    if (lane == 0) {
      const int my = (warp == 1) ? 0 : 1;
      long long it = 0, acc_it = 0;
      tc::RingPhases ring;   // this issuer's phases on its set, full[my][.]
      bool ok = true;
      for (long long t = blockIdx.x; t < total && ok && !*abort; t += gridDim.x) {
        const MultiTile m = multi_tile(jobs, t);
        const BcdJob &J = jobs.job[m.j];
        const int nk = J.Kp / kChunk;
        const uint32_t idesc = idesc_cols(m.R0, J.N);
        for (int v = J.v0; v < J.v1 && ok; ++v, ++acc_it) {
          const int buf = (int)(acc_it & 1);
          const uint32_t aph = (uint32_t)((acc_it >> 1) & 1);
          ok = tc::mbar_wait(&bar->acc_empty[buf], aph ^ 1u, limit, abort, jobs.status, 2);
          if (!ok) break;
          tc::tc_fence_after();
          {   // this issuer's chunks, at the ring positions bc_pos gives
            const int half = my;
            const uint32_t acc = tmem + buf * 256 + half * 128;
            for (int kc = 0; kc < nk; ++kc) {
              const int s = (int)((it + tc::bc_pos(kc, my, nk, nk)) % kStages);
              ok = tc::mbar_wait(&bar->full[my][s], ring.take(my, s), limit, abort, jobs.status, 4);
              if (!ok) break;
              tc::tc_fence_after();
              issue_chunk(acc, stage_ptr(smem, s, 0), kc == 0, chunk_steps(kc, J.n), idesc);
              tc::mma_commit(&bar->empty[s]);
            }
          }
          it += 2 * nk;
          if (ok) tc::mma_commit(&bar->acc_full[buf]);
        }
      }
      tc::mma_commit(&bar->drain);
      for (long long i = 0; i < wind_down_limit(limit) && !tc::mbar_try_wait(&bar->drain, 0); ++i) {
      }
    }
  } else if (warp >= 2 && warp <= 5) {
    // ---------------- epilogue: D[P, R] += B_v * C_v in registers ----------------
    const int q = warp & 3;
    const int row = q * 32 + lane;
    long long acc_it = 0;
    for (long long t = blockIdx.x; t < total && !*abort; t += gridDim.x) {
      const MultiTile m = multi_tile(jobs, t);
      const BcdJob &J = jobs.job[m.j];
      float d[kTile];
#pragma unroll
      for (int j = 0; j < kTile; ++j) d[j] = 0.f;
      bool ok = true;
      for (int v = J.v0; v < J.v1; ++v, ++acc_it) {
        const int buf = (int)(acc_it & 1);
        const uint32_t aph = (uint32_t)((acc_it >> 1) & 1);
        ok = tc::mbar_wait(&bar->acc_full[buf], aph, limit, abort, jobs.status, 8);
        if (!ok) break;
        tc::tc_fence_after();
        const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + buf * 256;
#pragma unroll
        for (int c = 0; c < kTile; c += 16) {
          float bv[16], cv[16];
          tc::tmem_ld_32x32b_x16(base + c, bv);
          tc::tmem_ld_32x32b_x16(base + 128 + c, cv);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 16; ++j) d[c + j] = fmaf(bv[j], cv[j], d[c + j]);
        }
        tc::tc_fence_before();
        tc::mbar_arrive(&bar->acc_empty[buf]);
      }
      if (!ok) break;
      const int P = m.P0 + row;
      if (P < J.N) {
        const float rs = J.row_scale[(long long)m.b * J.N + P];
        float *out = J.Dt + (long long)m.b * J.N * J.ldD + P;
#pragma unroll
        for (int j = 0; j < kTile; ++j) {
          const int R = m.R0 + j;
          if (R < J.N) out[(long long)R * J.ldD] = d[j] * rs * J.col_scale[(long long)m.b * J.N + R];
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

// ============================================================================
// Resident-operand variant of the fused kernel for Kp <= 128.  The per-tile
// operands G_Rq[R-tile] and G_wP^T[P-tile] (hi/lo, all of K) stay in shared
// memory for the whole tile (128 KB); only A_v and U2_v stream, one hi/lo chunk
// (32 KB) per stage.  That halves the bytes each MMA needs from L2, which is
// what limits the all-streamed kernel.
// ============================================================================
constexpr int kRStages = 3;
constexpr int kRStageBytes = 2 * kTileBytes;        // hi + lo of one 64-wide chunk
constexpr int kResBytes = 8 * kTileBytes;           // {GR, GW} x {hi, lo} x 2 chunks

struct ResBarriers {
  uint64_t full[2][kRStages];   // one set per MMA issuer, as in Barriers
  uint64_t empty[kRStages];
  uint64_t res_full, res_empty;
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

// resident tile address: op 0 = GR, 1 = GW; part 0 = hi, 1 = lo; chunk kc
__device__ __forceinline__ uint8_t *res_ptr(uint8_t *res, int op, int part, int kc) {
  return res + (size_t)((op * 2 + part) * 2 + kc) * kTileBytes;
}

template <int KS>
__device__ __forceinline__ void issue_chunk4_ks(uint32_t acc, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
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
__device__ __forceinline__ void issue_chunk4(uint32_t acc, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                             uint32_t b_lo, bool first, int ks, uint32_t idesc) {
  if (ks >= 4) issue_chunk4_ks<4>(acc, a_hi, a_lo, b_hi, b_lo, first, idesc);
  else if (ks == 3) issue_chunk4_ks<3>(acc, a_hi, a_lo, b_hi, b_lo, first, idesc);
  else if (ks == 2) issue_chunk4_ks<2>(acc, a_hi, a_lo, b_hi, b_lo, first, idesc);
  else issue_chunk4_ks<1>(acc, a_hi, a_lo, b_hi, b_lo, first, idesc);
}

__global__ void __launch_bounds__(kBcdThreads, 1)
    k_sox_bcd_tc_res(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
                     const __grid_constant__ CUtensorMap tmGR_hi, const __grid_constant__ CUtensorMap tmGR_lo,
                     const __grid_constant__ CUtensorMap tmGW_hi, const __grid_constant__ CUtensorMap tmGW_lo,
                     const __grid_constant__ CUtensorMap tmU_hi, const __grid_constant__ CUtensorMap tmU_lo,
                     BcdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *res = smem;
  uint8_t *stages = smem + kResBytes;
  ResBarriers *bar = reinterpret_cast<ResBarriers *>(stages + kRStages * kRStageBytes);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tP = (a.N + kTile - 1) / kTile;
  const int tiles_per_b = tP * tP;
  const long long total = (long long)a.batch * tiles_per_b;
  const int nk = a.Kp / kChunk;   // 1 or 2

  if (threadIdx.x == 0) {
    for (int s = 0; s < kRStages; ++s) {
      tc::mbar_init(&bar->full[0][s], 1);
      tc::mbar_init(&bar->full[1][s], 1);
      tc::mbar_init(&bar->empty[s], 1);
    }
    tc::mbar_init(&bar->res_full, 1);
    tc::mbar_init(&bar->res_empty, 2);   // one commit per issuing warp
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bar->acc_full[b], 2);
      tc::mbar_init(&bar->acc_empty[b], kEpiThreads);
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

  if (warp == 0) {
    if (lane == 0) {
      long long it = 0;
      tc::RingPhases ring;
      long long tt = 0;
      for (long long t = blockIdx.x; t < total && !*abort; t += gridDim.x, ++tt) {
        const int b = (int)(t / tiles_per_b);
        const int r = (int)(t % tiles_per_b);
        const int P0 = (r / tP) * kTile, R0 = (r % tP) * kTile;
        // resident operands of this tile, once the previous tile's MMAs are done with them
        if (!tc::mbar_wait(&bar->res_empty, (uint32_t)((tt & 1) ^ 1), a.spin_limit, abort, a.status, 16)) break;
        tc::mbar_arrive_expect_tx(&bar->res_full, (uint32_t)(4 * nk * kTileBytes));
        for (int kc = 0; kc < nk; ++kc) {
          const int x = kc * kChunk;
          tc::tma_load_3d(res_ptr(res, 0, 0, kc), &tmGR_hi, &bar->res_full, x, R0, b);
          tc::tma_load_3d(res_ptr(res, 0, 1, kc), &tmGR_lo, &bar->res_full, x, R0, b);
          tc::tma_load_3d(res_ptr(res, 1, 0, kc), &tmGW_hi, &bar->res_full, x, P0, b);
          tc::tma_load_3d(res_ptr(res, 1, 1, kc), &tmGW_lo, &bar->res_full, x, P0, b);
        }
        for (int v = a.v0; v < a.v1 && !*abort; ++v) {
          for (int p = 0; p < 2 * nk && !*abort; ++p, ++it) {
            int kc, half;
            tc::bc_decode(p, nk, 1, kc, half);
            const int s = (int)(it % kRStages);
            const uint32_t ph = (uint32_t)((it / kRStages) & 1);
            if (!tc::mbar_wait(&bar->empty[s], ph ^ 1u, a.spin_limit, abort, a.status, 1)) break;
            uint64_t *fb = &bar->full[half][s];
            ring.take(half, s);
            tc::mbar_arrive_expect_tx(fb, kRStageBytes);
            uint8_t *st = stages + (size_t)s * kRStageBytes;
            const int x = kc * kChunk;
            if (half == 0) {
              tc::tma_load_3d(st, &tmA_hi, fb, x, P0, b * a.n + v);
              tc::tma_load_3d(st + kTileBytes, &tmA_lo, fb, x, P0, b * a.n + v);
            } else {
              tc::tma_load_3d(st, &tmU_hi, fb, x, R0, v);
              tc::tma_load_3d(st + kTileBytes, &tmU_lo, fb, x, R0, v);
            }
          }
        }
      }
      // wind down: every stage issued must have landed before the CTA exits
      tc::ring_wind_down(bar->full, ring, wind_down_limit(a.spin_limit));
      if (tt > 0) {
        const uint32_t ph = (uint32_t)((tt - 1) & 1);
        for (long long i = 0; i < wind_down_limit(a.spin_limit) && !tc::mbar_try_wait(&bar->res_full, ph); ++i) {
        }
      }
    }
  } else if (warp == 1 || warp == 6) {
    // MMA issuers: warp 1 the B_v chunks, warp 6 the C_v chunks
    if (lane == 0) {
      const int my = (warp == 1) ? 0 : 1;
      long long it = 0, acc_it = 0;
      tc::RingPhases ring;   // this issuer's phases on its set, full[my][.]
      long long tt = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < total && ok && !*abort; t += gridDim.x, ++tt) {
        const uint32_t idesc = idesc_cols((int)((t % tiles_per_b) % tP) * kTile, a.N);   // R side
        ok = tc::mbar_wait(&bar->res_full, (uint32_t)(tt & 1), a.spin_limit, abort, a.status, 32);
        if (!ok) break;
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
              const int s = (int)((it + tc::bc_pos(kc, my, nk, 1)) % kRStages);
              ok = tc::mbar_wait(&bar->full[my][s], ring.take(my, s), a.spin_limit, abort, a.status, 4);
              if (!ok) break;
              tc::tc_fence_after();
              const uint32_t sh = smem_u32(stages + (size_t)s * kRStageBytes), sl = sh + kTileBytes;
              if (half == 0) {   // B_v[P, R] = A_v[P, :] . GR[R, :]
                issue_chunk4(acc, sh, sl, smem_u32(res_ptr(res, 0, 0, kc)), smem_u32(res_ptr(res, 0, 1, kc)), kc == 0,
                             chunk_steps(kc, a.n), idesc);
              } else {           // C_v[P, R] = GW[P, :] . U2_v[R, :]
                issue_chunk4(acc, smem_u32(res_ptr(res, 1, 0, kc)), smem_u32(res_ptr(res, 1, 1, kc)), sh, sl, kc == 0,
                             chunk_steps(kc, a.n), idesc);
              }
              tc::mma_commit(&bar->empty[s]);
            }
          }
          it += 2 * nk;
          if (ok) tc::mma_commit(&bar->acc_full[buf]);
        }
        if (ok) tc::mma_commit(&bar->res_empty);   // resident tiles free once these MMAs retire
      }
      tc::mma_commit(&bar->drain);
      for (long long i = 0; i < wind_down_limit(a.spin_limit) && !tc::mbar_try_wait(&bar->drain, 0); ++i) {
      }
    }
  } else if (warp >= 2 && warp <= 5) {
    bcd_epilogue(bar, tmem, a, tP, total, abort, warp, lane);
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ============================================================================
// Pair variant of the fused kernel: two CTAs on neighbouring SMs share every MMA
// (tcgen05 cta_group::2, M = 256 over the pair, N = 128).  A work unit is (batch b,
// a pair of 128-row P tiles, one 128-column R tile); each CTA owns one P tile (its
// A_v / G_wP^T rows, its TMEM rows of B_v and C_v, its rows of D) and loads HALF of
// the shared R-side operand (G_Rq or U2_v rows R0 + 64 rank .. +64).  Per SM every
// MMA reads 128 + 64 operand rows from shared memory instead of 128 + 128, and the
// copies into shared memory shrink by the same quarter.  The even CTA issues the
// MMAs; both CTAs' copies of a stage complete on the even CTA's `full` barrier, the
// MMA commits arrive on both CTAs' `empty` / `acc_full` barriers, and both CTAs'
// epilogue warps release an accumulator buffer on the even CTA's `acc_empty`.
// An odd P-tile count leaves the odd CTA of the last pair on rows >= N (loaded as
// zeros, never written).
// ============================================================================
constexpr int kPStages = 4;
constexpr int kPATile = kTile * kChunk * 2;               // 128 rows x 64 K, FP16: 16 KB
constexpr int kPBTile = (kTile / 2) * kChunk * 2;         // 64 rows: 8 KB
constexpr int kPStageBytes = 2 * kPATile + 2 * kPBTile;   // A hi/lo + B-half hi/lo: 48 KB
constexpr uint32_t kPairIdesc = tc::idesc_f16_f32(2 * kTile, kTile);

struct PairBarriers {
  uint64_t full[2][kPStages]; // even CTA: both CTAs' copies of a stage have landed (one set per issuer)
  uint64_t empty[kPStages];   // each CTA: the pair's MMAs are done with its copy of a stage
  uint64_t acc_full[2];       // each CTA: B_v and C_v of an accumulator buffer are complete
  uint64_t acc_empty[2];      // even CTA: the 8 epilogue warps of the pair have read a buffer
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

template <int KS>
__device__ __forceinline__ void issue_chunk_pair_ks(uint32_t acc, uint32_t st, bool first) {
  const uint32_t a_hi = st, a_lo = st + kPATile, b_hi = st + 2 * kPATile, b_lo = b_hi + kPBTile;
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const uint32_t off = k * 32;
    tc::mma_f16_pair(acc, tc::desc_kmajor_sw128(a_hi + off), tc::desc_kmajor_sw128(b_lo + off), kPairIdesc,
                     (first && k == 0) ? 0u : 1u);
    tc::mma_f16_pair(acc, tc::desc_kmajor_sw128(a_lo + off), tc::desc_kmajor_sw128(b_hi + off), kPairIdesc, 1u);
  }
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const uint32_t off = k * 32;
    tc::mma_f16_pair(acc, tc::desc_kmajor_sw128(a_hi + off), tc::desc_kmajor_sw128(b_hi + off), kPairIdesc, 1u);
  }
}
__device__ __forceinline__ void issue_chunk_pair(uint32_t acc, uint32_t st, bool first, int ks) {
  if (ks >= 4) issue_chunk_pair_ks<4>(acc, st, first);
  else if (ks == 3) issue_chunk_pair_ks<3>(acc, st, first);
  else if (ks == 2) issue_chunk_pair_ks<2>(acc, st, first);
  else issue_chunk_pair_ks<1>(acc, st, first);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kBcdThreads, 1)
    k_sox_bcd_pair(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
                   const __grid_constant__ CUtensorMap tmGR_hi, const __grid_constant__ CUtensorMap tmGR_lo,
                   const __grid_constant__ CUtensorMap tmGW_hi, const __grid_constant__ CUtensorMap tmGW_lo,
                   const __grid_constant__ CUtensorMap tmU_hi, const __grid_constant__ CUtensorMap tmU_lo,
                   BcdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  PairBarriers *bar = reinterpret_cast<PairBarriers *>(smem + kPStages * kPStageBytes);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t rank = tc::cluster_ctarank();   // 0: the CTA that issues the pair's MMAs
  const long long pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int tP = (a.N + kTile - 1) / kTile;
  const int tPP = (tP + 1) / 2;
  const long long units_per_b = (long long)tPP * tP;
  const long long total = (long long)a.batch * units_per_b;
  const int nk = a.Kp / kChunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kPStages; ++s) {
      tc::mbar_init(&bar->full[0][s], 1);
      tc::mbar_init(&bar->full[1][s], 1);
      tc::mbar_init(&bar->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bar->acc_full[b], 2);   // one multicast commit per issuing warp
      tc::mbar_init(&bar->acc_empty[b], 8);
    }
    tc::mbar_init(&bar->drain, 2);
    bar->abort = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc_pair(&bar->tmem_base, 512);
    tc::tmem_relinquish_pair();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmA_hi); tc::prefetch_tmap(&tmA_lo); tc::prefetch_tmap(&tmGR_hi);
    tc::prefetch_tmap(&tmGR_lo); tc::prefetch_tmap(&tmGW_hi); tc::prefetch_tmap(&tmGW_lo);
    tc::prefetch_tmap(&tmU_hi); tc::prefetch_tmap(&tmU_lo);
  }
  // both CTAs' barriers initialised (and TMEM allocated) before either CTA touches the other's
  tc::tc_fence_before();
  tc::cluster_sync();
  tc::tc_fence_after();
  const uint32_t tmem = bar->tmem_base;
  volatile int *abort = &bar->abort;
  const uint32_t full0 = tc::mapa_shared(tc::smem_u32(&bar->full[0][0]), 0);   // full[q][s]: + (q S + s) 8
  const uint32_t acc_empty0 = tc::mapa_shared(tc::smem_u32(&bar->acc_empty[0]), 0);

  if (warp == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    if (lane == 0) {
      long long it = 0;
      tc::RingPhases ring;
      for (long long u = pair; u < total && !*abort; u += npairs) {
        const int b = (int)(u / units_per_b);
        const int r = (int)(u % units_per_b);
        const int P0 = (2 * (r / tP) + (int)rank) * kTile;
        const int R0 = (r % tP) * kTile + (int)rank * (kTile / 2);
        for (int v = a.v0; v < a.v1 && !*abort; ++v) {
          for (int p = 0; p < 2 * nk && !*abort; ++p, ++it) {
            int kc, half;
            tc::bc_decode(p, nk, 1, kc, half);
            const int s = (int)(it % kPStages);
            const uint32_t ph = (uint32_t)((it / kPStages) & 1);
            if (!tc::mbar_wait(&bar->empty[s], ph ^ 1u, a.spin_limit, abort, a.status, 1)) break;
            ring.take(half, s);   // the half's issuer
            if (rank == 0) tc::mbar_arrive_expect_tx(&bar->full[half][s], 2 * kPStageBytes);
            const uint32_t fb = full0 + (uint32_t)(half * kPStages + s) * 8u;
            uint8_t *st = smem + (size_t)s * kPStageBytes;
            const int x = kc * kChunk;
            if (half == 0) {   // B_v = A_v . GR^T
              tc::tma_load_3d_pair(st, &tmA_hi, fb, x, P0, b * a.n + v);
              tc::tma_load_3d_pair(st + kPATile, &tmA_lo, fb, x, P0, b * a.n + v);
              tc::tma_load_3d_pair(st + 2 * kPATile, &tmGR_hi, fb, x, R0, b);
              tc::tma_load_3d_pair(st + 2 * kPATile + kPBTile, &tmGR_lo, fb, x, R0, b);
            } else {           // C_v = G_wP^T . U2_v^T
              tc::tma_load_3d_pair(st, &tmGW_hi, fb, x, P0, b);
              tc::tma_load_3d_pair(st + kPATile, &tmGW_lo, fb, x, P0, b);
              tc::tma_load_3d_pair(st + 2 * kPATile, &tmU_hi, fb, x, R0, v);
              tc::tma_load_3d_pair(st + 2 * kPATile + kPBTile, &tmU_lo, fb, x, R0, v);
            }
          }
        }
      }
      // wind down (even CTA): every stage issued by either CTA has landed
      if (rank == 0) tc::ring_wind_down(bar->full, ring, wind_down_limit(a.spin_limit));
    }
  } else if (warp == 1 || warp == 6) {
    // ---------------- MMA issuers (even CTA): warp 1 the B_v chunks, warp 6 the C_v chunks ----------------
    if (lane == 0 && rank == 0) {
      const int my = (warp == 1) ? 0 : 1;
      long long it = 0, acc_it = 0;
      tc::RingPhases ring;   // this issuer's phases on its set, full[my][.]
      bool ok = true;
      for (long long u = pair; u < total && ok && !*abort; u += npairs) {
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
              const int s = (int)((it + tc::bc_pos(kc, my, nk, 1)) % kPStages);
              ok = tc::mbar_wait(&bar->full[my][s], ring.take(my, s), a.spin_limit, abort, a.status, 4);
              if (!ok) break;
              tc::tc_fence_after();
              issue_chunk_pair(acc, tc::smem_u32(smem + (size_t)s * kPStageBytes), kc == 0, chunk_steps(kc, a.n));
              tc::mma_commit_pair_mc(&bar->empty[s], 3);
            }
          }
          it += 2 * nk;
          if (ok) tc::mma_commit_pair_mc(&bar->acc_full[buf], 3);
        }
      }
      // all MMAs complete before TMEM is released
      tc::mma_commit_pair(&bar->drain);
      for (long long i = 0; i < wind_down_limit(a.spin_limit) && !tc::mbar_try_wait(&bar->drain, 0); ++i) {
      }
    }
  } else if (warp >= 2 && warp <= 5) {
    // ---------------- epilogue (both CTAs): D[P, R] += B_v * C_v in registers ----------------
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int row = q * 32 + lane;          // P offset inside this CTA's tile
    long long acc_it = 0;
    for (long long u = pair; u < total && !*abort; u += npairs) {
      const int b = (int)(u / units_per_b);
      const int r = (int)(u % units_per_b);
      const int P0 = (2 * (r / tP) + (int)rank) * kTile, R0 = (r % tP) * kTile;
      float d[kTile];
#pragma unroll
      for (int j = 0; j < kTile; ++j) d[j] = 0.f;
      bool ok = true;
      for (int v = a.v0; v < a.v1; ++v, ++acc_it) {
        const int buf = (int)(acc_it & 1);
        const uint32_t aph = (uint32_t)((acc_it >> 1) & 1);
        ok = tc::mbar_wait(&bar->acc_full[buf], aph, a.spin_limit, abort, a.status, 8);
        if (!ok) break;
        tc::tc_fence_after();
        const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + buf * 256;
#pragma unroll
        for (int c = 0; c < kTile; c += 16) {
          float bv[16], cv[16];
          tc::tmem_ld_32x32b_x16(base + c, bv);
          tc::tmem_ld_32x32b_x16(base + 128 + c, cv);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 16; ++j) d[c + j] = fmaf(bv[j], cv[j], d[c + j]);
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive_cluster(acc_empty0 + (uint32_t)buf * 8u);
      }
      if (!ok) break;
      const int P = P0 + row;
      if (P < a.N) {
        const float rs = a.row_scale[(long long)b * a.N + P];
        float *out = a.Dt + (long long)b * a.N * a.ldD + P;
#pragma unroll
        for (int j = 0; j < kTile; ++j) {
          const int R = R0 + j;
          if (R < a.N) out[(long long)R * a.ldD] = d[j] * rs * a.col_scale[(long long)b * a.N + R];
        }
      }
    }
  }
  // neither CTA leaves (or frees TMEM) while the other may still read its shared memory
  // or arrive on its barriers
  __syncwarp();
  tc::tc_fence_before();
  tc::cluster_sync();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc_pair(tmem, 512);
  }
}

// ============================================================================
// Split GEMM with split output (the A intermediate, Sec. II C):
//   C[b](i, j) = sum_k A[bA](i, k) B[bB](j, k)      (both operands K-major FP16 pairs)
// 128 x 128 tiles, double-buffered TMEM accumulator.  The epilogue scales the
// tile (kStoreSplit: out_scale[b]; kStoreSplitGroup: an exact power of two per
// group of `group` columns, all of whose rows lie in the tile), splits it into
// FP16 pairs in swizzled shared memory and writes it with TMA tensor stores into
// the 4-D output [batch][M][n_groups][group] (box: 128 rows x 64 columns).
// ============================================================================
constexpr int kGStages = 2;
constexpr int kStageOut = 4 * kTile * 64 * 2;   // hi/lo x two 64-column halves, 64 KB

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, const void *src, int x, int y, int z, int w) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z), "r"(w)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// The split GEMM runs 8 epilogue warps (two per TMEM lane quarter, one per
// 64-column half): the epilogue, not the MMA, sets its pace.
// warp 0 TMA, warps 1 and 10 MMA (even and odd tiles of the CTA, one issuing while the other
// waits for a stage), warps 2-9 epilogue
constexpr int kGemmThreads = 352;
constexpr int kGemmEpi = 256;
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// the epilogue warps agree on ok (all of them, or none, go on: no warp is left waiting at a
// named barrier that the others have stopped reaching)
__device__ __forceinline__ bool epi_all(bool ok) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((unsigned)ok)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int x, int y, int z) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
               : "memory");
}
// element-wise FP32 add of the shared tile into global memory (round to nearest)
__device__ __forceinline__ void tma_reduce_add_3d(const CUtensorMap *map, const void *src, int x, int y, int z) {
  asm volatile("cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
               : "memory");
}
// Output tile t of a GEMM launch: batch b and the tile's first row i0 and column j0.  When
// every batch shares one B operand (no index table), the column tiles go slowest, then the
// batches, then the row tiles, so all the tiles that read one B tile run one after another
// and B leaves DRAM once per launch (the A GEMM of the chain: U_Pqs of up to 0.7 GB read
// by every (tau, row tile) pair would otherwise be re-read from DRAM for each); otherwise
// batches slowest, then rows, then columns.
struct GemmTile {
  int b, i0, j0;
};
__device__ __forceinline__ GemmTile gemm_tile(const GemmTcArgs &a, long long t, int tM, int tN) {
  GemmTile g;
  if (a.batchB_shared && !a.idxB) {
    const long long per_j = (long long)a.batch * tM;
    const long long j = t / per_j, r = t % per_j;
    g.b = (int)(r / tM);
    g.i0 = (int)(r % tM) * kTile;
    g.j0 = (int)j * kTile;
  } else {
    const long long per_b = (long long)tM * tN;
    const long long r = t % per_b;
    g.b = (int)(t / per_b);
    g.i0 = (int)(r / tN) * kTile;
    g.j0 = (int)(r % tN) * kTile;
  }
  return g;
}

// kStoreF32 scale of tile t for epilogue thread e: e < 128 the column scale of tile column e,
// else alpha times the row scale of tile row e - 128
__device__ __forceinline__ float f32_tile_scale(const GemmTcArgs &a, long long t, int e, int tM, int tN) {
  const GemmTile g = gemm_tile(a, t, tM, tN);
  const int b = g.b;
  if (e < kTile) {
    const int col = g.j0 + e;
    if (!a.col_scale || col >= a.Ncols) return 1.f;
    const int zb = a.idxB ? a.idxB[b] : (a.batchB_shared ? 0 : b);
    return a.col_scale[zb * a.cs_b + col];
  }
  const int row = g.i0 + (e - kTile);
  if (!a.row_scale || row >= a.M) return a.alpha;
  const int za = a.idxA ? a.idxA[b] : (a.batchA_shared ? 0 : b);
  return a.alpha * a.row_scale[za * a.rs_b + row];
}

__device__ __forceinline__ uint32_t pack2(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_f16x2(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
                 const __grid_constant__ CUtensorMap tmB_hi, const __grid_constant__ CUtensorMap tmB_lo,
                 const __grid_constant__ CUtensorMap tmC_hi, const __grid_constant__ CUtensorMap tmC_lo,
                 GemmTcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *stage_out = smem + kGStages * kStageBytes;
  Barriers *bar = reinterpret_cast<Barriers *>(stage_out + kStageOut);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tM = (a.M + kTile - 1) / kTile, tN = (a.Ncols + kTile - 1) / kTile;
  const long long per_b = (long long)tM * tN;
  const long long total = per_b * a.batch;
  const int nk = a.Kp / kChunk;
  const int kv = (a.K > 0 && a.K < a.Kp) ? a.K : a.Kp;   // valid K (the rest is zero padding)

  setup_barriers(bar, kGemmEpi);
  if (warp == 1) {
    tc::tmem_alloc(&bar->tmem_base, 256);
    tc::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmA_hi); tc::prefetch_tmap(&tmA_lo);
    tc::prefetch_tmap(&tmB_hi); tc::prefetch_tmap(&tmB_lo);
    tc::prefetch_tmap(&tmC_hi); tc::prefetch_tmap(&tmC_lo);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = bar->tmem_base;
  volatile int *abort = &bar->abort;

  if (warp == 0) {
    if (lane == 0) {
      long long it = 0, tt = 0;
      tc::RingPhases ring;
      for (long long t = blockIdx.x; t < total && !*abort; t += gridDim.x, ++tt) {
        const int q = (int)(tt & 1);   // issuer of this tile
        const GemmTile gt = gemm_tile(a, t, tM, tN);
        const int b = gt.b, i0 = gt.i0, j0 = gt.j0;
        const int za = a.idxA ? a.idxA[b] : (a.batchA_shared ? 0 : b);
        const int zb = a.idxB ? a.idxB[b] : (a.batchB_shared ? 0 : b);
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = (int)(it % kGStages);
          const uint32_t ph = (uint32_t)((it / kGStages) & 1);
          if (!tc::mbar_wait(&bar->empty[s], ph ^ 1u, a.spin_limit, abort, a.status, 1)) break;
          uint64_t *fb = &bar->full[q][s];
          ring.take(q, s);
          tc::mbar_arrive_expect_tx(fb, kStageBytes);
          const int x = kc * kChunk;
          tc::tma_load_3d(stage_ptr(smem, s, 0), &tmA_hi, fb, x, i0, za);
          tc::tma_load_3d(stage_ptr(smem, s, 1), &tmA_lo, fb, x, i0, za);
          tc::tma_load_3d(stage_ptr(smem, s, 2), &tmB_hi, fb, x, j0, zb);
          tc::tma_load_3d(stage_ptr(smem, s, 3), &tmB_lo, fb, x, j0, zb);
        }
      }
      tc::ring_wind_down(bar->full, ring, wind_down_limit(a.spin_limit));
    }
  } else if (warp == 1 || warp == 10) {
    if (lane == 0) {
      const long long my = (warp == 1) ? 0 : 1;
      long long it = 0, acc_it = 0;
      tc::RingPhases ring;   // this issuer's phases on its set, full[my][.]
      bool ok = true;
      for (long long t = blockIdx.x; t < total && ok && !*abort; t += gridDim.x, ++acc_it) {
        if ((acc_it & 1) != my) {   // the other issuer's tile
          it += nk;
          continue;
        }
        const int buf = (int)(acc_it & 1);
        const uint32_t aph = (uint32_t)((acc_it >> 1) & 1);
        ok = tc::mbar_wait(&bar->acc_empty[buf], aph ^ 1u, a.spin_limit, abort, a.status, 2);
        if (!ok) break;
        tc::tc_fence_after();
        const uint32_t acc = tmem + buf * 128;
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = (int)(it % kGStages);
          ok = tc::mbar_wait(&bar->full[my][s], ring.take((int)my, s), a.spin_limit, abort, a.status, 4);
          if (!ok) break;
          tc::tc_fence_after();
          issue_chunk(acc, stage_ptr(smem, s, 0), kc == 0, chunk_steps(kc, kv));
          tc::mma_commit(&bar->empty[s]);
        }
        if (ok) tc::mma_commit(&bar->acc_full[buf]);
      }
      tc::mma_commit(&bar->drain);
      for (long long i = 0; i < wind_down_limit(a.spin_limit) && !tc::mbar_try_wait(&bar->drain, 0); ++i) {
      }
    }
  } else if (warp <= 9) {
    const int q = warp & 3;
    const int row = q * 32 + lane;          // tile row = TMEM lane
    const int h = (warp - 2) >> 2;          // 64-column half of the tile
    const bool storer = (warp == 2 && lane == 0);
    __shared__ float red[8];
    __shared__ __align__(16) float s_sc[2 * kTile];   // kStoreF32: column scales, then alpha x row scales
    const int ep = (warp - 2) * 32 + lane;
    // the scales of the next tile are loaded one tile ahead (their latency hides behind this one)
    float pre = (a.mode == kStoreF32 && blockIdx.x < total) ? f32_tile_scale(a, blockIdx.x, ep, tM, tN) : 0.f;
    long long acc_it = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x, ++acc_it) {
      const GemmTile gt = gemm_tile(a, t, tM, tN);
      const int b = gt.b, i0 = gt.i0, j0 = gt.j0;
      const int buf = (int)(acc_it & 1);
      const uint32_t aph = (uint32_t)((acc_it >> 1) & 1);
      const bool got = tc::mbar_wait(&bar->acc_full[buf], aph, a.spin_limit, abort, a.status, 8);
      if (!epi_all(got && !*abort)) break;
      tc::tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + buf * 128 + h * 64;
      const bool row_ok = (i0 + row) < a.M;
      if (a.mode == kStoreF32) {
        // scaled FP32 tile in four 128-byte-swizzled boxes of 128 rows x 32 columns, written
        // (or added, in accumulate mode) by TMA tensor stores; rows >= M and columns >= Ncols
        // fall outside the tensor map and are not written
        if (storer) bulk_wait_read();   // the previous tile's stores have read the staging boxes
        epi_sync();
        s_sc[ep] = pre;
        epi_sync();
        if (t + gridDim.x < total) pre = f32_tile_scale(a, t + gridDim.x, ep, tM, tN);
        const float rsc = s_sc[kTile + row];
        float *tile = reinterpret_cast<float *>(stage_out);
#pragma unroll
        for (int c = 0; c < 64; c += 32) {
          float v[32];
          tc::tmem_ld_32x32b_x32(base + c, v);
          tc::tmem_ld_wait();
          if (c == 32) {
            tc::tc_fence_before();
            tc::mbar_arrive(&bar->acc_empty[buf]);
          }
          const int col = h * 64 + c;    // tile column of v[0]; box col / 32 holds v[0..31]
          float *box = tile + (col / 32) * (kTile * 32) + row * 32;
#pragma unroll
          for (int t4 = 0; t4 < 8; ++t4) {
            const float4 cs = *reinterpret_cast<const float4 *>(&s_sc[col + 4 * t4]);
            *reinterpret_cast<float4 *>(box + ((t4 ^ (row & 7)) * 4)) =
                make_float4(v[4 * t4] * (rsc * cs.x), v[4 * t4 + 1] * (rsc * cs.y), v[4 * t4 + 2] * (rsc * cs.z),
                            v[4 * t4 + 3] * (rsc * cs.w));
          }
        }
        fence_proxy_async_smem();
        epi_sync();
        if (storer) {
#pragma unroll
          for (int bx = 0; bx < 4; ++bx) {
            const int x = j0 + 32 * bx;
            if (x < a.Ncols) {
              if (a.accumulate)
                tma_reduce_add_3d(&tmC_hi, stage_out + (size_t)bx * (kTile * 128), x, i0, b);
              else
                tma_store_3d(&tmC_hi, stage_out + (size_t)bx * (kTile * 128), x, i0, b);
            }
          }
          bulk_commit();
        }
        continue;
      }
      // this half's columns belong to group g (groups are 64 or 128 columns wide)
      const int g = (h * 64) >= a.group ? 1 : 0;
      float sc = 1.f;
      if (a.mode == kStoreSplit) {
        sc = a.out_scale[b];
      } else {
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < 64; c += 32) {
          float v[32];
          tc::tmem_ld_32x32b_x32(base + c, v);
          tc::tmem_ld_wait();
          if (row_ok) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) m = fmaxf(m, fabsf(v[jj]));
          }
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) red[warp - 2] = m;
        epi_sync();
        float mg = 0.f;
#pragma unroll
        for (int w2 = 0; w2 < 8; ++w2) {
          const int g2 = ((w2 >> 2) * 64) >= a.group ? 1 : 0;
          if (g2 == g) mg = fmaxf(mg, red[w2]);
        }
        sc = tc::pow2_floor_inv(mg);
        if (q == 0 && lane == 0 && (g == h)) {   // one writer per group: warp of quarter 0, half g
          const int grp = (j0 + h * 64) / a.group;
          if (grp < a.n_groups) a.group_scale[(long long)b * a.n_groups + grp] = sc;
        }
      }
      // the previous tile's TMA stores must have read the staging buffer
      if (storer) bulk_wait_read();
      epi_sync();
      // split into FP16 pairs, written to the 128-byte-swizzled staging tile of this half
      uint8_t *hi_tile = stage_out + (size_t)(0 * 2 + h) * (kTile * 128);
      uint8_t *lo_tile = stage_out + (size_t)(1 * 2 + h) * (kTile * 128);
#pragma unroll
      for (int c = 0; c < 64; c += 32) {
        float v[32];
        tc::tmem_ld_32x32b_x32(base + c, v);
        tc::tmem_ld_wait();
        if (c == 32) {  // this half of the accumulator is read: hand it back
          tc::tc_fence_before();
          tc::mbar_arrive(&bar->acc_empty[buf]);
        }
#pragma unroll
        for (int t16 = 0; t16 < 4; ++t16) {
          uint32_t ph[4], pl[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int jj = t16 * 8 + e * 2;
            __half h0, l0, h1, l1;
            tc::split_f16(v[jj] * sc, h0, l0);
            tc::split_f16(v[jj + 1] * sc, h1, l1);
            ph[e] = pack2(h0, h1);
            pl[e] = pack2(l0, l1);
          }
          const int chunk = (c / 8 + t16) ^ (row & 7);
          *reinterpret_cast<uint4 *>(hi_tile + row * 128 + chunk * 16) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
          *reinterpret_cast<uint4 *>(lo_tile + row * 128 + chunk * 16) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
        }
      }
      fence_proxy_async_smem();
      epi_sync();
      if (storer) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int col = j0 + hh * 64;
          if (col < a.Ncols) {
            const int grp = col / a.group, x = col % a.group;
            tma_store_4d(&tmC_hi, stage_out + (size_t)(0 * 2 + hh) * (kTile * 128), x, grp, i0, b);
            tma_store_4d(&tmC_lo, stage_out + (size_t)(1 * 2 + hh) * (kTile * 128), x, grp, i0, b);
          }
        }
        bulk_commit();
      }
    }
    if (storer) bulk_wait_all();
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 256);
  }
}

// ------------------------------- split helpers ------------------------------

__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One warp per output row: hi/lo of src row scaled to max in [1, 2); rows >= rows_valid are zero.
__global__ void k_split_rows_f64(const double *src, long long ld, long long bstride, int rows_valid,
                                 int rows_out, int L, int Kp, __half *hi, __half *lo, float *inv_scale,
                                 int batch, const double *alt_src, const int *use_alt) {
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (gw >= (long long)rows_out * batch) return;
  const int b = (int)(gw / rows_out), r = (int)(gw % rows_out);
  __half *h = hi + ((long long)b * rows_out + r) * Kp;
  __half *l = lo + ((long long)b * rows_out + r) * Kp;
  if (r >= rows_valid) {
    for (int k = lane; k < Kp; k += 32) h[k] = l[k] = __float2half(0.f);
    return;
  }
  const double *x = ((use_alt && use_alt[b]) ? alt_src : src) + b * bstride + r * ld;
  float m = 0.f;
  for (int k = lane; k < L; k += 32) m = fmaxf(m, (float)fabs(x[k]));
  m = warp_max(m);
  const float s = tc::pow2_floor_inv(m);
  for (int k = lane; k < Kp; k += 32) {
    __half a = __float2half(0.f), c = __float2half(0.f);
    if (k < L) {
      // scale in FP64 (exact: power of two), then round to the FP16 pair via FP32
      const double xs = x[k] * (double)s;
      const float f = (float)xs;
      a = __float2half_rn(f);
      c = __float2half_rn((float)(xs - (double)__half2float(a)));
    }
    h[k] = a;
    l[k] = c;
  }
  if (lane == 0 && inv_scale) inv_scale[(long long)b * rows_valid + r] = 1.f / s;
}

__device__ float block_max(float v) {
  __shared__ float red[32];
  v = warp_max(v);
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x / 32) ? red[lane] : 0.f;
    v = warp_max(v);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  return red[0];
}

// Mixed tensor U[P][q][s] (FP32, Kp x Kp per P) -> split with one scale per P, written as
//   U1 layout [P][q][s]     (if u1_hi)   and/or   U2 layout [v][R][w] = U[R][v][w] (if u2_hi, v < n,
//   R-stride NR rows)
__global__ void k_split_mixed(const float *U, int N, int NR, int n, int Kp, __half *u1_hi, __half *u1_lo,
                              __half *u2_hi, __half *u2_lo, float *inv_scale) {
  const int P = blockIdx.x;
  const long long blk = (long long)Kp * Kp;
  const float *u = U + (long long)P * blk;
  float m = 0.f;
  for (long long e = threadIdx.x; e < blk; e += blockDim.x) m = fmaxf(m, fabsf(u[e]));
  m = block_max(m);
  const float s = tc::pow2_floor_inv(m);
  for (long long e = threadIdx.x; e < blk; e += blockDim.x) {
    __half hi, lo;
    tc::split_f16(u[e] * s, hi, lo);
    if (u1_hi) {
      u1_hi[(long long)P * blk + e] = hi;
      u1_lo[(long long)P * blk + e] = lo;
    }
    const int v = (int)(e / Kp), w = (int)(e % Kp);
    if (u2_hi && v < n) {
      const long long o = ((long long)v * NR + P) * Kp + w;
      u2_hi[o] = hi;
      u2_lo[o] = lo;
    }
  }
  if (threadIdx.x == 0) inv_scale[P] = 1.f / s;
}

// Per batch b (spin, tau): Gm = G(-tau) = -G[T-1-j] as Gm^T[v][s] split with one scale
// g = 2^-floor(log2 max|Gm|); out_scale = 2^-ceil(log2(2 max_v sum_s |g Gm[s][v]|)) bounds
// the A products so their split stays in FP16 range.
__global__ void k_prep_gminus(const double *G, int n, int T, int Kp, __half *hi, __half *lo,
                              float *gscale, float *out_scale, int b0, int rows_out) {
  const int b = blockIdx.x;
  const int sp = (b0 + b) / T, j = (b0 + b) % T;
  const double *g = G + ((long long)sp * T + (T - 1 - j)) * n * n;
  float m = 0.f;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) m = fmaxf(m, (float)fabs(g[e]));
  m = block_max(m);
  const float sc = tc::pow2_floor_inv(m);
  float cs = 0.f;
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    float acc = 0.f;
    for (int s = 0; s < n; ++s) acc += (float)fabs(g[(long long)s * n + v]) * sc;
    cs = fmaxf(cs, acc);
  }
  cs = block_max(cs) * 2.f * 1.0001f;
  // 2^-ceil(log2 cs)
  int e;
  const float f = frexpf(cs, &e);  // cs = f 2^e, f in [0.5, 1)
  const float os = ldexpf(1.f, (f == 0.5f) ? -(e - 1) : -e);
  __half *h = hi + (long long)b * rows_out * Kp;
  __half *l = lo + (long long)b * rows_out * Kp;
  for (int e2 = threadIdx.x; e2 < rows_out * Kp; e2 += blockDim.x) {
    const int v = e2 / Kp, s = e2 % Kp;
    __half a = __float2half(0.f), c = __float2half(0.f);
    if (v < n && s < n) {
      const double xs = -g[(long long)s * n + v] * (double)sc;
      a = __float2half_rn((float)xs);
      c = __float2half_rn((float)(xs - (double)__half2float(a)));
    }
    h[e2] = a;
    l[e2] = c;
  }
  if (threadIdx.x == 0) {
    gscale[b] = sc;
    out_scale[b] = os;
  }
}

// row/col factors of the fused kernel's output:
//   row[b][P] = inv_u1[P] / (g[b] o[b]) * inv_gw[b][P],   col[b][R] = inv_gr[b][R] * inv_u2[R]
__global__ void k_bcd_scales(const float *inv_u1, const float *gsc, const float *osc, const float *asc,
                             int NR, const float *inv_gw, const float *inv_gr, const float *inv_u2, int N,
                             int batch, float *row, float *col) {
  const long long total = (long long)N * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / N), P = (int)(e % N);
    const double a_sc = asc ? asc[(long long)b * NR + P] : osc[b];
    // products of up to four clamped powers of two: form them in FP64 and clamp
    // into the normal FP32 range (a factor outside it only scales values that
    // are themselves outside FP32 range, i.e. zero at any tolerance)
    const double r = (double)inv_u1[P] / ((double)gsc[b] * a_sc) * (double)inv_gw[e];
    const double c = (double)inv_gr[e] * (double)inv_u2[P];
    row[e] = (float)fmin(fmax(r, 0x1p-126), 0x1p126);
    col[e] = (float)fmin(fmax(c, 0x1p-126), 0x1p126);
  }
}

// Mixed THC tensor U[P][q][s] = sum_Q V[P][Q] X[Q][q] X[Q][s] (Eq. U_contraction at k = 0),
// FP32 round-to-nearest accumulation over Q on CUDA cores; columns (q, s) run over
// the padded Kp x Kp block and are zero outside [0, n)^2.  64 x 64 tile, 4 x 4 per thread.
__global__ void __launch_bounds__(256) k_mixed_f32(const double *V, const double *X, int N, int n, int Kp,
                                                   float *U) {
  __shared__ float sa[16][65];
  __shared__ float sb[16][65];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int P0 = blockIdx.y * 64;
  const long long c0 = (long long)blockIdx.x * 64;
  const long long ncol = (long long)Kp * Kp;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < N; k0 += 16) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int e = tid + it * 256;
      const int rr = e / 16, kk = e % 16;
      const int P = P0 + rr, Q = k0 + kk;
      sa[kk][rr] = (P < N && Q < N) ? (float)V[(long long)P * N + Q] : 0.f;
      const int kb = e / 64, cc = e % 64;
      const int Qb = k0 + kb;
      const long long col = c0 + cc;
      const int q = (int)(col / Kp), sidx = (int)(col % Kp);
      sb[kb][cc] = (Qb < N && col < ncol && q < n && sidx < n)
                       ? (float)(X[(long long)Qb * n + q] * X[(long long)Qb * n + sidx])
                       : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = sa[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = sb[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int P = P0 + ty + 16 * i;
    if (P >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long col = c0 + tx + 16 * j;
      if (col < ncol) U[(long long)P * ncol + col] = acc[i][j];
    }
  }
}

// T[b][R][r] = sum_P Dt[b][R][P] X[P][r]   (FP32 accumulate; D carries FP32 accuracy)
// 64 x 64 tile of (R, r) per block, 256 threads, 4 x 4 per thread.
__global__ void __launch_bounds__(256) k_backproject_T(const float *Dt, long long ldD, const double *X, int N,
                                                       int n, float *T) {
  __shared__ float sa[16][65];
  __shared__ float sb[16][65];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int R0 = blockIdx.y * 64, r0 = blockIdx.x * 64;
  const int b = blockIdx.z;
  const float *D = Dt + (long long)b * N * ldD;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < N; k0 += 16) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int e = tid + it * 256;
      const int rr = e / 16, kk = e % 16;
      const int R = R0 + rr, P = k0 + kk;
      sa[kk][rr] = (R < N && P < N) ? D[(long long)R * ldD + P] : 0.f;
      const int kb = e / 64, cc = e % 64;
      const int Pb = k0 + kb, c = r0 + cc;
      sb[kb][cc] = (Pb < N && c < n) ? (float)X[(long long)Pb * n + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = sa[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = sb[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int R = R0 + ty + 16 * i;
    if (R >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = r0 + tx + 16 * j;
      if (c < n) T[((long long)b * N + R) * n + c] = acc[i][j];
    }
  }
}

// Sigma[b][t][r] = -sum_R X[R][t] T[b][R][r]   (FP64 accumulate: the final orbital-basis sum)
__global__ void __launch_bounds__(256) k_backproject_sigma(const double *X, const float *T, int N, int n,
                                                           double *Sigma, long long sstride, const int *sym) {
  __shared__ double sa[16][33];
  __shared__ double sb[16][33];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int t0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int b = blockIdx.z;
  // symmetric Sigma (bare SOX, symmetric G): lower-triangle blocks are mirrored by the upper ones
  const bool mirror = sym && sym[b];
  if (mirror && blockIdx.y > blockIdx.x) return;
  const float *Tb = T + (long long)b * N * n;
  double acc[2][2] = {};
  for (int k0 = 0; k0 < N; k0 += 16) {
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int e = tid + it * 256;
      const int kk = e / 32, cc = e % 32;
      const int R = k0 + kk;
      sa[kk][cc] = (R < N && t0 + cc < n) ? X[(long long)R * n + t0 + cc] : 0.0;
      sb[kk][cc] = (R < N && c0 + cc < n) ? (double)Tb[(long long)R * n + c0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const double a0 = sa[kk][ty], a1 = sa[kk][ty + 16];
      const double b0 = sb[kk][tx], b1 = sb[kk][tx + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int t = t0 + ty + 16 * i;
    if (t >= n) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < n) {
        Sigma[(long long)b * sstride + (long long)t * n + c] = -acc[i][j];
        if (mirror && blockIdx.y < blockIdx.x) Sigma[(long long)b * sstride + (long long)c * n + t] = -acc[i][j];
      }
    }
  }
}

}  // namespace

// ------------------------------ launchers ----------------------------------

void launch_mixed_f32(const double *V, const double *X, int N, int n, int Kp, float *U, cudaStream_t s) {
  const long long ncol = (long long)Kp * Kp;
  dim3 grid((unsigned)((ncol + 63) / 64), (N + 63) / 64);
  k_mixed_f32<<<grid, 256, 0, s>>>(V, X, N, n, Kp, U);
}

void launch_backproject_T(const float *Dt, long long ldD, const double *X, int N, int n, int batch, float *T,
                          cudaStream_t s) {
  dim3 grid((n + 63) / 64, (N + 63) / 64, batch);
  k_backproject_T<<<grid, 256, 0, s>>>(Dt, ldD, X, N, n, T);
}

void launch_backproject_sigma(const double *X, const float *T, int N, int n, int batch, double *Sigma,
                              long long sstride, cudaStream_t s, const int *sym) {
  dim3 grid((n + 31) / 32, (n + 31) / 32, batch);
  k_backproject_sigma<<<grid, 256, 0, s>>>(X, T, N, n, Sigma, sstride, sym);
}

size_t tc_smem_bytes() { return (size_t)kStages * kStageBytes + sizeof(Barriers) + 1024; }

size_t res_smem_bytes() { return (size_t)kResBytes + kRStages * kRStageBytes + sizeof(ResBarriers) + 1024; }

size_t pair_smem_bytes() { return (size_t)kPStages * kPStageBytes + sizeof(PairBarriers) + 1024; }

// How many CTA pairs of the pair kernel fit on the device at once (queried once per device).
cudaError_t pair_capacity(int *pairs) {
  static std::atomic<int> cache[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int c = cache[dev & 63].load();
  if (c > 0) {
    *pairs = c;
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2, 1, 1);
  cfg.blockDim = dim3(kBcdThreads, 1, 1);
  cfg.dynamicSmemBytes = pair_smem_bytes();
  int n = 0;
  e = cudaOccupancyMaxActiveClusters(&n, k_sox_bcd_pair, &cfg);
  if (e != cudaSuccess) return e;
  if (n < 1) return cudaErrorInvalidConfiguration;
  cache[dev & 63].store(n);
  *pairs = n;
  return cudaSuccess;
}

cudaError_t launch_sox_bcd_tc(const CUtensorMap *maps, const BcdArgs &args, int grid, cudaStream_t s, int variant) {
  BcdArgs a = args;
  a.v1 = (a.v1 <= 0 || a.v1 > a.n) ? a.n : a.v1;
  a.v0 = a.v0 < 0 ? 0 : (a.v0 > a.v1 ? a.v1 : a.v0);
  if (variant == kBcdResident && a.Kp <= 128) {
    static std::atomic<unsigned long long> rattr{0};
    const cudaError_t e = set_smem_once(k_sox_bcd_tc_res, (int)res_smem_bytes(), rattr);
    if (e != cudaSuccess) return e;
    k_sox_bcd_tc_res<<<grid, kBcdThreads, res_smem_bytes(), s>>>(maps[0], maps[1], maps[2], maps[3], maps[4],
                                                               maps[5], maps[6], maps[7], a);
    return cudaGetLastError();
  }
  if (variant == kBcdPair) {
    static std::atomic<unsigned long long> pattr{0};
    cudaError_t e = set_smem_once(k_sox_bcd_pair, (int)pair_smem_bytes(), pattr);
    if (e != cudaSuccess) return e;
    int pairs = 0;
    e = pair_capacity(&pairs);
    if (e != cudaSuccess) return e;
    const int tP = (a.N + kTile - 1) / kTile;
    const long long units = (long long)a.batch * ((tP + 1) / 2) * tP;
    const int g = 2 * (int)std::max<long long>(1, std::min<long long>(units, pairs));
    k_sox_bcd_pair<<<g, kBcdThreads, pair_smem_bytes(), s>>>(maps[0], maps[1], maps[8], maps[9], maps[4], maps[5],
                                                            maps[10], maps[11], a);
    return cudaGetLastError();
  }
  static std::atomic<unsigned long long> attr{0};
  const cudaError_t e = set_smem_once(k_sox_bcd_tc, (int)tc_smem_bytes(), attr);
  if (e != cudaSuccess) return e;
  k_sox_bcd_tc<<<grid, kBcdThreads, tc_smem_bytes(), s>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5],
                                                        maps[6], maps[7], a);
  return cudaGetLastError();
}

cudaError_t launch_sox_bcd_multi(const BcdJobs &jobs, int grid, cudaStream_t s) {
  if (jobs.count <= 0 || jobs.count > kMaxBcdJobs) return cudaErrorInvalidValue;
  if (jobs.total <= 0) return cudaSuccess;
  static std::atomic<unsigned long long> attr{0};
  const cudaError_t e = set_smem_once(k_sox_bcd_multi, (int)tc_smem_bytes(), attr);
  if (e != cudaSuccess) return e;
  k_sox_bcd_multi<<<grid, kBcdThreads, tc_smem_bytes(), s>>>(jobs);
  return cudaGetLastError();
}

size_t gemm_smem_bytes() { return (size_t)kGStages * kStageBytes + kStageOut + sizeof(Barriers) + 1024; }

cudaError_t launch_gemm_f16x2(const CUtensorMap *maps, const GemmTcArgs &a, int grid, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  const cudaError_t e = set_smem_once(k_gemm_f16x2, (int)gemm_smem_bytes(), attr);
  if (e != cudaSuccess) return e;
  k_gemm_f16x2<<<grid, kGemmThreads, gemm_smem_bytes(), s>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], a);
  return cudaGetLastError();
}

bool make_tmap_f16_store4d(CUtensorMap *map, const void *base, uint64_t group, uint64_t n_groups, uint64_t rows,
                           uint64_t batch, std::string *err) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      if (err) *err = "cuTensorMapEncodeTiled entry point not available";
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  // element (x, grp, row, b) at ((b * rows + row) * n_groups + grp) * group + x
  cuuint64_t dims[4] = {group, n_groups, rows, batch};
  cuuint64_t strides[3] = {group * 2, group * n_groups * 2, group * n_groups * rows * 2};
  cuuint32_t box[4] = {64, 1, 128, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void *>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled (store) failed with CUresult " + std::to_string((int)r);
    return false;
  }
  return true;
}

bool make_tmap_f32_store3d(CUtensorMap *map, const void *base, uint64_t cols, uint64_t rows, uint64_t batch,
                           uint64_t ld, uint64_t batch_stride, std::string *err) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      if (err) *err = "cuTensorMapEncodeTiled entry point not available";
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  // element (x, row, b) at b * batch_stride + row * ld + x; box 32 columns (128 B) x 128 rows
  cuuint64_t dims[3] = {cols, rows, batch};
  cuuint64_t strides[2] = {ld * 4, batch_stride * 4};
  cuuint32_t box[3] = {32, 128, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled (FP32 store) failed with CUresult " + std::to_string((int)r);
    return false;
  }
  return true;
}

void launch_split_rows_f64(const double *src, long long ld, long long bstride, int rows_valid, int rows_out,
                           int L, int Kp, __half *hi, __half *lo, float *inv_scale, int batch, cudaStream_t s,
                           const double *alt_src, const int *use_alt) {
  const long long warps = (long long)rows_out * batch;
  const int blocks = (int)((warps * 32 + 255) / 256);
  k_split_rows_f64<<<blocks, 256, 0, s>>>(src, ld, bstride, rows_valid, rows_out, L, Kp, hi, lo, inv_scale,
                                          batch, alt_src, use_alt);
}

void launch_split_mixed(const float *U, int N, int NR, int n, int Kp, __half *u1_hi, __half *u1_lo,
                        __half *u2_hi, __half *u2_lo, float *inv_scale, cudaStream_t s) {
  k_split_mixed<<<N, 256, 0, s>>>(U, N, NR, n, Kp, u1_hi, u1_lo, u2_hi, u2_lo, inv_scale);
}

void launch_prep_gminus(const double *G, int n, int T, int nbatch, int Kp, __half *hi, __half *lo,
                        float *gscale, float *out_scale, int b0, int rows_out, cudaStream_t s) {
  // batches b0 .. b0+nbatch-1 of the flattened (spin, tau) index; outputs indexed from 0
  k_prep_gminus<<<nbatch, 256, 0, s>>>(G, n, T, Kp, hi, lo, gscale, out_scale, b0, rows_out);
}

void launch_bcd_scales(const float *inv_u1, const float *gsc, const float *osc, const float *asc, int NR,
                       const float *inv_gw, const float *inv_gr, const float *inv_u2, int N, int batch,
                       float *row, float *col, cudaStream_t s) {
  const long long total = (long long)N * batch;
  k_bcd_scales<<<(int)std::min<long long>((total + 255) / 256, 65535), 256, 0, s>>>(
      inv_u1, gsc, osc, asc, NR, inv_gw, inv_gr, inv_u2, N, batch, row, col);
}

}  // namespace sox
