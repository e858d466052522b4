// Split-precision GEMM on tcgen05 with FP32 output and operands in either shared-memory
// major order, plus per-tensor FP16-pair splits.
//
// Why MN-major: the reverse pass of Phi (Sec. II C chain run backwards) contracts the
// same tensors over different indices -- Bbar_v[P][R] over R (rows P) and over P (rows
// R), A_v[P][q] over q and over P.  A K-major-only GEMM needs a transposed copy of each
// such tensor; with the MMA reading an MN-major tile (instruction-descriptor transpose
// bit, 64-element MN blocks of 128-byte swizzled rows) one stored layout serves both.
// That needs one scale per tensor (a per-row scale would vary along K in one of the
// two uses), hence the per-tensor splits below: every tensor is scaled by a power of
// two that puts its largest entry in [2^14, 2^15), so entries down to 2^-17 of the
// largest keep the full 22 bits of the (hi, lo) pair and smaller ones an absolute error
// of 2^-25 (FP16 subnormal spacing) -- far below the FP32-class bound of the sums.
#include <algorithm>
#include <atomic>

#include "gemm_mn.h"
#include "smem_attr.h"
#include "tc_common.cuh"

namespace sox {

using tc::smem_u32;

namespace {

constexpr int kT = 128;                       // tile rows / columns
constexpr int kC = 64;                        // K elements per chunk
constexpr int kPart = kT * kC * 2;            // 16 KB: hi (or lo) of one operand for one chunk
constexpr int kStageBytes = 4 * kPart;        // A hi, A lo, B hi, B lo
constexpr int kStages = 3;
constexpr int kOutBytes = kT * 64 * 4;        // FP32 staging of one 64-column half of an output tile
// warp 0 TMA, warps 1 and 10 MMA, warps 2-9 epilogue; eleven warps take the registers of
// twelve, as ten do.  The accumulation windows of an item go two at a time, their chunks
// alternating in the stage ring, the even window issued by warp 1 and the odd one by warp
// 10: one issuer keeps the tensor pipe fed while the other waits for a stage.  Four TMEM
// accumulators (window w in buffer w % 4) let a pair accumulate while the epilogue drains
// the previous pair.
constexpr int kThreads = 352;
constexpr int kEpi = 256;

// full[q][s]: stage s holds a chunk of an accumulation window of issuer q.  Each issuer
// waits only on its own set, so the phases it counts are the ones it consumes (an issuer
// that skipped the other's window would otherwise wait on a phase two ahead of the
// barrier, where the parity test already reads as complete).
struct Bars {
  uint64_t full[2][kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[4];    // window w accumulates in TMEM buffer w % 4
  uint64_t acc_empty[4];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ long long wind_down(long long cap) { return cap > (1LL << 20) ? cap : (1LL << 20); }

// MN-major shared-memory descriptor, 128-byte swizzle: rows of 128 bytes hold 64
// consecutive MN elements for one k, 8 rows (k .. k+7) form a 1024-byte atom (SBO), and
// the second 64-element MN block of the 128-wide tile starts `lbo` bytes further.
__device__ __forceinline__ uint64_t desc_mn_sw128(uint32_t saddr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ uint64_t op_desc(uint32_t base, int mn, int k16) {
  // K step of 16: 32 bytes along a K-major row, or 16 rows (2 atoms, 2048 bytes) MN-major
  return mn ? desc_mn_sw128(base + k16 * 2048, kPart / 2) : tc::desc_kmajor_sw128(base + k16 * 32);
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
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
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int x, int y, int z) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
               : "memory");
}
__device__ __forceinline__ void tma_reduce_add_3d(const CUtensorMap *map, const void *src, int x, int y, int z) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

struct Item {
  int b, i0, j0;
  long long c0, c1;   // chunk range
};

// work item t -> (batch, split, tile row, tile column); tile columns run fastest so
// items in flight together share their A chunks through L2
__device__ __forceinline__ Item item_of(const GemmMnArgs &a, long long t, int tM, int tN, long long total) {
  Item it;
  const long long tiles = (long long)tM * tN;
  const long long per_b = tiles * a.ksplit;
  it.b = (int)(t / per_b);
  long long r = t % per_b;
  const long long ks = r / tiles;
  r %= tiles;
  it.i0 = (int)(r / tN) * kT;
  it.j0 = (int)(r % tN) * kT;
  it.c0 = ks * a.cps;
  it.c1 = it.c0 + a.cps < total ? it.c0 + a.cps : total;
  return it;
}

__device__ __forceinline__ void load_operand(uint8_t *dst, const CUtensorMap *hi, const CUtensorMap *lo, uint64_t *bar,
                                             int mn, int row0, int k0, int z) {
  if (mn) {
    tc::tma_load_3d(dst, hi, bar, row0, k0, z);
    tc::tma_load_3d(dst + kPart / 2, hi, bar, row0 + 64, k0, z);
    tc::tma_load_3d(dst + kPart, lo, bar, row0, k0, z);
    tc::tma_load_3d(dst + kPart + kPart / 2, lo, bar, row0 + 64, k0, z);
  } else {
    tc::tma_load_3d(dst, hi, bar, k0, row0, z);
    tc::tma_load_3d(dst + kPart, lo, bar, k0, row0, z);
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_mn(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
              const __grid_constant__ CUtensorMap tmB_hi, const __grid_constant__ CUtensorMap tmB_lo,
              const __grid_constant__ CUtensorMap tmC, GemmMnArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *stage_out = smem + kStages * kStageBytes;
  Bars *bar = reinterpret_cast<Bars *>(stage_out + kOutBytes);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tM = (a.M + kT - 1) / kT, tN = (a.Ncols + kT - 1) / kT;
  const long long chunks = (long long)a.kc_inner * a.nk_outer;
  const long long items = (long long)a.batch * tM * tN * a.ksplit;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&bar->full[0][s], 1);
      tc::mbar_init(&bar->full[1][s], 1);
      tc::mbar_init(&bar->empty[s], 1);
    }
    for (int b = 0; b < 4; ++b) {
      tc::mbar_init(&bar->acc_full[b], 1);
      tc::mbar_init(&bar->acc_empty[b], kEpi);
    }
    tc::mbar_init(&bar->drain, 2);   // one commit per issuing warp
    bar->abort = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(&bar->tmem_base, 512);
    tc::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmA_hi); tc::prefetch_tmap(&tmA_lo);
    tc::prefetch_tmap(&tmB_hi); tc::prefetch_tmap(&tmB_lo);
    tc::prefetch_tmap(&tmC);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = bar->tmem_base;
  volatile int *abort = &bar->abort;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      long long it = 0, acc0 = 0;   // acc0: windows of the previous items
      tc::RingPhases ring;
      for (long long t = blockIdx.x; t < items && !*abort; t += gridDim.x) {
        const Item w = item_of(a, t, tM, tN, chunks);
        // the item's windows two at a time, their chunks alternating in the ring
        for (long long p0 = w.c0; p0 < w.c1 && !*abort; p0 += 2 * a.window) {
          const long long L0 = w.c1 - p0 < a.window ? w.c1 - p0 : a.window;
          const long long r1 = w.c1 - p0 - a.window;
          const long long L1 = r1 <= 0 ? 0 : (r1 < a.window ? r1 : a.window);
          const long long wi = acc0 + (p0 - w.c0) / a.window;   // the pair's first window
          for (long long i = 0; i < L0 && !*abort; ++i) {
            for (int hh = 0; hh < 2 && (hh == 0 || i < L1); ++hh, ++it) {
              const int s = (int)(it % kStages);
              const uint32_t ph = (uint32_t)((it / kStages) & 1);
              if (!tc::mbar_wait(&bar->empty[s], ph ^ 1u, a.spin_limit, abort, a.status, 1)) break;
              const int q = (int)((wi + hh) & 1);   // issuer of the chunk's window
              uint64_t *fb = &bar->full[q][s];
              ring.take(q, s);
              tc::mbar_arrive_expect_tx(fb, kStageBytes);
              const long long c = p0 + hh * a.window + i;
              const long long kz = c / a.kc_inner;
              const int k0 = (int)(c % a.kc_inner) * kC;
              uint8_t *st = smem + (size_t)s * kStageBytes;
              load_operand(st, &tmA_hi, &tmA_lo, fb, a.a.mn_major, w.i0, k0,
                           (int)(a.a.z0 + (w.b / a.a.zdiv) * a.a.zb + kz * a.a.zk));
              load_operand(st + 2 * kPart, &tmB_hi, &tmB_lo, fb, a.b.mn_major, w.j0, k0,
                           (int)(a.b.z0 + (w.b / a.b.zdiv) * a.b.zb + kz * a.b.zk));
            }
          }
        }
        if (w.c1 > w.c0) acc0 += (w.c1 - w.c0 + a.window - 1) / a.window;
      }
      // every copy issued has landed before the CTA exits
      tc::ring_wind_down(bar->full, ring, wind_down(a.spin_limit));
    }
  } else if (warp == 1 || warp == 10) {
    // ---------------- MMA issuers: warp 1 the even windows, warp 10 the odd ones ----------------
    if (lane == 0) {
      const long long my = (warp == 1) ? 0 : 1;
      long long it = 0, acc_it = 0;
      tc::RingPhases ring;   // this issuer's phases on its set, full[my][.]
      bool ok = true;
      for (long long t = blockIdx.x; t < items && ok && !*abort; t += gridDim.x) {
        const Item w = item_of(a, t, tM, tN, chunks);
        // N = the tile's valid columns rounded up to 16: no MMA over the zero rows of B past Ncols
        const int wN = a.Ncols - w.j0 >= kT ? kT : ((a.Ncols - w.j0 + 15) & ~15);
        const uint32_t idesc = tc::idesc_f16_f32(kT, wN) | ((uint32_t)a.a.mn_major << 15) |
                               ((uint32_t)a.b.mn_major << 16);
        for (long long p0 = w.c0; p0 < w.c1 && ok; p0 += 2 * a.window) {
          const long long L0 = w.c1 - p0 < a.window ? w.c1 - p0 : a.window;
          const long long r1 = w.c1 - p0 - a.window;
          const long long L1 = r1 <= 0 ? 0 : (r1 < a.window ? r1 : a.window);
          const int hh = (int)((my - acc_it) & 1);   // this issuer's window of the pair: acc_it + hh
          const long long Lh = hh ? L1 : L0;
          if (Lh > 0) {
            const long long wi = acc_it + hh;
            const int buf = (int)(wi & 3);
            const uint32_t aph = (uint32_t)((wi >> 2) & 1);
            ok = tc::mbar_wait(&bar->acc_empty[buf], aph ^ 1u, a.spin_limit, abort, a.status, 2);
            if (!ok) break;
            tc::tc_fence_after();
            const uint32_t acc = tmem + buf * kT;
            for (long long i = 0; i < Lh; ++i) {
              // ring position of chunk i: the pair alternates while both windows have chunks
              const long long pos = it + (i < L1 ? 2 * i + hh : 2 * L1 + (i - L1));
              const int s = (int)(pos % kStages);
              ok = tc::mbar_wait(&bar->full[my][s], ring.take((int)my, s), a.spin_limit, abort, a.status, 4);
              if (!ok) break;
              tc::tc_fence_after();
              const uint32_t st = smem_u32(smem + (size_t)s * kStageBytes);
              const uint32_t ahi = st, alo = st + kPart, bhi = st + 2 * kPart, blo = st + 3 * kPart;
              const bool first = (i == 0);
              // the small cross terms first, the large hi*hi steps last (truncating accumulation)
#pragma unroll
              for (int k = 0; k < kC / 16; ++k) {
                tc::mma_f16(acc, op_desc(ahi, a.a.mn_major, k), op_desc(blo, a.b.mn_major, k), idesc,
                            (first && k == 0) ? 0u : 1u);
                tc::mma_f16(acc, op_desc(alo, a.a.mn_major, k), op_desc(bhi, a.b.mn_major, k), idesc, 1u);
              }
#pragma unroll
              for (int k = 0; k < kC / 16; ++k)
                tc::mma_f16(acc, op_desc(ahi, a.a.mn_major, k), op_desc(bhi, a.b.mn_major, k), idesc, 1u);
              tc::mma_commit(&bar->empty[s]);
            }
            if (ok) tc::mma_commit(&bar->acc_full[buf]);
          }
          it += L0 + L1;
          acc_it += L1 > 0 ? 2 : 1;
        }
      }
      tc::mma_commit(&bar->drain);
      for (long long i = 0; i < wind_down(a.spin_limit) && !tc::mbar_try_wait(&bar->drain, 0); ++i) {
      }
    }
  } else if (warp <= 9) {
    // ---------------- epilogue: 8 warps, lane quarter q, 64-column half h ----------------
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int h = (warp - 2) >> 2;
    const bool storer = (warp == 2 && lane == 0);
    const float alpha = a.alpha_host * (a.alpha ? *a.alpha : 1.f);
    long long acc_it = 0;
    bool live = true;
    for (long long t = blockIdx.x; t < items && live; t += gridDim.x) {
      const Item w = item_of(a, t, tM, tN, chunks);
      float sum[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) sum[j] = 0.f;
      for (long long w0 = w.c0; w0 < w.c1; w0 += a.window, ++acc_it) {
        const int buf = (int)(acc_it & 3);
        const uint32_t aph = (uint32_t)((acc_it >> 2) & 1);
        const bool got = tc::mbar_wait(&bar->acc_full[buf], aph, a.spin_limit, abort, a.status, 8);
        if (!epi_all(got && !*abort)) {
          live = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + buf * kT + h * 64;
#pragma unroll
        for (int c = 0; c < 64; c += 32) {
          float v[32];
          tc::tmem_ld_32x32b_x32(base + c, v);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 32; ++j) sum[c + j] += v[j];
        }
        tc::tc_fence_before();
        tc::mbar_arrive(&bar->acc_empty[buf]);
      }
      if (!live) break;
      // scaled tile -> TMA, one 64-column half at a time through the staging buffer (two
      // 128-byte-swizzled boxes of 128 rows x 32 columns); the half-h warps fill it
      float *tile = reinterpret_cast<float *>(stage_out);
      const bool add = a.accumulate || a.ksplit > 1;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        if (storer) bulk_wait_read();   // the previous stores have read the staging buffer
        epi_sync();
        if (h == half) {
#pragma unroll
          for (int c = 0; c < 64; c += 32) {
            float *box = tile + (c / 32) * (kT * 32) + row * 32;
#pragma unroll
            for (int t4 = 0; t4 < 8; ++t4)
              *reinterpret_cast<float4 *>(box + ((t4 ^ (row & 7)) * 4)) =
                  make_float4(sum[c + 4 * t4] * alpha, sum[c + 4 * t4 + 1] * alpha, sum[c + 4 * t4 + 2] * alpha,
                              sum[c + 4 * t4 + 3] * alpha);
          }
        }
        fence_proxy_async_smem();
        epi_sync();
        if (storer) {
#pragma unroll
          for (int bx = 0; bx < 2; ++bx) {
            const int x = w.j0 + half * 64 + 32 * bx;
            if (x < a.Ncols) {
              if (add)
                tma_reduce_add_3d(&tmC, stage_out + (size_t)bx * (kT * 128), x, w.i0, w.b);
              else
                tma_store_3d(&tmC, stage_out + (size_t)bx * (kT * 128), x, w.i0, w.b);
            }
          }
          bulk_commit();
        }
      }
    }
    if (storer) bulk_wait_all();
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ------------------------------ per-tensor splits ------------------------------

// Work unit u of the per-tensor kernels: one warp, 256 consecutive columns (lane + 32 k,
// k < 8) of one row r = (r1, r0); the index divisions happen once per unit.
constexpr int kUnitCols = 256;

// |x| as FP32 (an FP64 value rounds up to at most one FP32 ulp); FP32 sources stay on the
// FP32 pipe (the FP64 rate is 1/64 of it)
__device__ __forceinline__ float abs_f(float x) { return fabsf(x); }
__device__ __forceinline__ float abs_f(double x) { return (float)fabs(x); }

// FP16 pair of x * sd (sd a signed power of two; x * sd exact): hi rounds to nearest and
// lo = RN(x sd - hi).  For an FP32 x both steps are exact in FP32, so no FP64 arithmetic
// is needed; an FP64 x keeps its remainder in FP64.
__device__ __forceinline__ void split_scaled(float x, float sf, double, __half &a, __half &b) {
  const float xs = x * sf;
  a = __float2half_rn(xs);
  b = __float2half_rn(xs - __half2float(a));
}
__device__ __forceinline__ void split_scaled(double x, float, double sd, __half &a, __half &b) {
  const double xs = x * sd;
  a = __float2half_rn((float)xs);
  b = __float2half_rn((float)(xs - (double)__half2float(a)));
}

template <class T>
__global__ void k_absmax(const T *src, long long ld0, int rows0, long long ld1, int rows1, long long ldc, int cols,
                         float *out) {
  const long long cpr = (cols + kUnitCols - 1) / kUnitCols;
  const long long units = (long long)rows1 * rows0 * cpr;
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  float m = 0.f;
  for (long long u = warp0; u < units; u += nwarps) {
    const long long r = u / cpr;
    const int c0 = (int)(u % cpr) * kUnitCols;
    const long long r1 = r / rows0, r0 = r % rows0;
    const T *row = src + r1 * ld1 + r0 * ld0;
#pragma unroll
    for (int k = 0; k < kUnitCols / 32; ++k) {
      const int c = c0 + lane + 32 * k;
      if (c < cols) m = fmaxf(m, abs_f(row[(long long)c * ldc]));
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  // non-negative floats order like their bit patterns
  if (lane == 0 && m > 0.f) atomicMax(reinterpret_cast<unsigned int *>(out), __float_as_uint(m));
}

// 2^(14 - floor(log2 m)) for m > 0 (m in [2^e, 2^(e+1)) -> scaled max in [2^14, 2^15)), 1 for
// m == 0; clamped to normal FP32 powers of two
__device__ __forceinline__ float big_scale(float m) {
  if (!(m > 0.f)) return 1.f;
  int e;
  frexpf(m, &e);   // m = f 2^e, f in [0.5, 1): floor(log2 m) = e - 1
  int k = 15 - e;
  k = k < -120 ? -120 : (k > 120 ? 120 : k);
  return ldexpf(1.f, k);
}

template <class T>
__global__ void k_split_tensor(const T *src, long long ld0, int rows0, long long ld1, int rows1, long long ldc,
                               int cols, long long ldo, long long ldo1, float sign, const float *absmax,
                               const float *scale_in, __half *hi, __half *lo, float *scale_out) {
  const float s = scale_in ? *scale_in : big_scale(*absmax);
  const double sd = (double)sign * (double)s;
  const float sf = sign * s;
  const long long cpr = (ldo + kUnitCols - 1) / kUnitCols;
  const long long units = (long long)rows1 * rows0 * cpr;
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long u = warp0; u < units; u += nwarps) {
    const long long r = u / cpr;
    const long long c0 = (u % cpr) * kUnitCols;
    const long long r1 = r / rows0, r0 = r % rows0;
    const T *row = src + r1 * ld1 + r0 * ld0;
    __half *h = hi + r1 * ldo1 + r0 * ldo, *l = lo + r1 * ldo1 + r0 * ldo;
#pragma unroll
    for (int k = 0; k < kUnitCols / 32; ++k) {
      const long long c = c0 + lane + 32 * k;
      if (c >= ldo) break;
      __half a = __float2half(0.f), b = __float2half(0.f);
      if (c < cols) split_scaled(row[c * ldc], sf, sd, a, b);
      h[c] = a;
      l[c] = b;
    }
  }
  if (scale_out && blockIdx.x == 0 && threadIdx.x == 0) *scale_out = s;
}

// FP32 rows with unit column stride, two columns per lane (8-byte loads, 4-byte stores):
// the same values as the kernels above, for rows whose starts are 8-byte aligned in the
// source and 4-byte aligned in the outputs.  A unit is 512 consecutive columns.
constexpr int kUnitCols2 = 512;

__global__ void k_absmax_f32x2(const float *src, long long ld0, int rows0, long long ld1, int rows1, int cols,
                               float *out) {
  const long long cpr = (cols + kUnitCols2 - 1) / kUnitCols2;
  const long long units = (long long)rows1 * rows0 * cpr;
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  float m = 0.f;
  for (long long u = warp0; u < units; u += nwarps) {
    const long long r = u / cpr;
    const int c0 = (int)(u % cpr) * kUnitCols2;
    const long long r1 = r / rows0, r0 = r % rows0;
    const float *row = src + r1 * ld1 + r0 * ld0;
#pragma unroll
    for (int k = 0; k < kUnitCols2 / 64; ++k) {
      const int c = c0 + 2 * lane + 64 * k;
      if (c + 1 < cols) {
        const float2 x = *reinterpret_cast<const float2 *>(row + c);
        m = fmaxf(m, fmaxf(fabsf(x.x), fabsf(x.y)));
      } else if (c < cols) {
        m = fmaxf(m, fabsf(row[c]));
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0 && m > 0.f) atomicMax(reinterpret_cast<unsigned int *>(out), __float_as_uint(m));
}

__global__ void k_split_f32x2(const float *src, long long ld0, int rows0, long long ld1, int rows1, int cols,
                              long long ldo, long long ldo1, float sign, const float *absmax, const float *scale_in,
                              __half *hi, __half *lo, float *scale_out) {
  const float s = scale_in ? *scale_in : big_scale(*absmax);
  const float sf = sign * s;
  const long long cpr = (ldo + kUnitCols2 - 1) / kUnitCols2;
  const long long units = (long long)rows1 * rows0 * cpr;
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long u = warp0; u < units; u += nwarps) {
    const long long r = u / cpr;
    const long long c0 = (u % cpr) * kUnitCols2;
    const long long r1 = r / rows0, r0 = r % rows0;
    const float *row = src + r1 * ld1 + r0 * ld0;
    __half *h = hi + r1 * ldo1 + r0 * ldo, *l = lo + r1 * ldo1 + r0 * ldo;
#pragma unroll
    for (int k = 0; k < kUnitCols2 / 64; ++k) {
      const long long c = c0 + 2 * lane + 64 * k;
      if (c >= ldo) break;   // ldo is even: c + 1 < ldo
      float2 x = make_float2(0.f, 0.f);
      if (c + 1 < cols) x = *reinterpret_cast<const float2 *>(row + c);
      else if (c < cols) x.x = row[c];
      uint32_t a, b;
      tc::split_f16x2(x.x * sf, x.y * sf, a, b);
      *reinterpret_cast<uint32_t *>(h + c) = a;
      *reinterpret_cast<uint32_t *>(l + c) = b;
    }
  }
  if (scale_out && blockIdx.x == 0 && threadIdx.x == 0) *scale_out = s;
}

// true when the FP32 two-column kernels apply: unit column stride, even row pitches and
// 8-byte (source) / 4-byte (outputs) aligned bases
bool f32x2_ok(const void *src, long long ld0, long long ld1, long long ldc) {
  return ldc == 1 && (ld0 % 2) == 0 && (ld1 % 2) == 0 && (reinterpret_cast<uintptr_t>(src) % 8) == 0;
}

// blocks of 256 threads (8 warps) for `units` warp-sized work units, at most 32 per SM
int blocks_for_units(long long units) {
  return (int)std::max<long long>(1, std::min<long long>((units + 7) / 8, 152 * 32));
}

}  // namespace

int plan_gemm_mn(GemmMnArgs &a, int sms, int max_ksplit) {
  const long long tiles = (long long)a.batch * ((a.M + kT - 1) / kT) * ((a.Ncols + kT - 1) / kT);
  const long long chunks = (long long)a.kc_inner * a.nk_outer;
  const long long windows = (chunks + a.window - 1) / a.window;
  // Items run in waves of `sms` (one CTA per SM, items strided over the grid); each costs
  // its windows plus about a quarter window of epilogue.  Pick the split with the least
  // modelled time: ceil(items / sms) x (windows per item + 1/4).
  long long best_ks = 1;
  double best = -1.0;
  const long long kmax = std::max<long long>(1, std::min<long long>(max_ksplit, windows));
  for (long long ks = 1; ks <= kmax; ++ks) {
    const long long wps = (windows + ks - 1) / ks;
    const long long split = (windows + wps - 1) / wps;
    const long long items = tiles * split;
    const double cost = (double)((items + sms - 1) / sms) * ((double)wps + 0.25);
    if (best < 0.0 || cost < best - 1e-9) {
      best = cost;
      best_ks = ks;
    }
  }
  const long long wps = (windows + best_ks - 1) / best_ks;   // windows per split item
  a.cps = wps * a.window;
  a.ksplit = (int)((chunks + a.cps - 1) / a.cps);            // every item has at least one chunk
  const long long items = tiles * a.ksplit;
  return (int)std::max<long long>(1, std::min<long long>(items, sms));
}

cudaError_t launch_gemm_mn(const CUtensorMap *maps, const GemmMnArgs &a, int grid, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  const int bytes = kStages * kStageBytes + kOutBytes + (int)sizeof(Bars) + 1024;
  const cudaError_t e = set_smem_once(k_gemm_mn, bytes, attr);
  if (e != cudaSuccess) return e;
  k_gemm_mn<<<grid, kThreads, bytes, s>>>(maps[0], maps[1], maps[2], maps[3], maps[4], a);
  return cudaGetLastError();
}

void launch_absmax(const void *src, bool f32, long long ld0, int rows0, long long ld1, int rows1, long long ldc,
                   int cols, float *out, cudaStream_t s) {
  if (f32 && f32x2_ok(src, ld0, ld1, ldc)) {
    const int blocks = blocks_for_units((long long)rows1 * rows0 * ((cols + kUnitCols2 - 1) / kUnitCols2));
    k_absmax_f32x2<<<blocks, 256, 0, s>>>(static_cast<const float *>(src), ld0, rows0, ld1, rows1, cols, out);
    return;
  }
  const int blocks = blocks_for_units((long long)rows1 * rows0 * ((cols + kUnitCols - 1) / kUnitCols));
  if (f32)
    k_absmax<float><<<blocks, 256, 0, s>>>(static_cast<const float *>(src), ld0, rows0, ld1, rows1, ldc, cols, out);
  else
    k_absmax<double><<<blocks, 256, 0, s>>>(static_cast<const double *>(src), ld0, rows0, ld1, rows1, ldc, cols, out);
}

void launch_split_tensor(const void *src, bool f32, long long ld0, int rows0, long long ld1, int rows1, long long ldc,
                         int cols, long long ldo, long long ldo1, float sign, const float *absmax,
                         const float *scale_in, __half *hi, __half *lo, float *scale_out, cudaStream_t s) {
  if (f32 && f32x2_ok(src, ld0, ld1, ldc) && (ldo % 2) == 0 && (ldo1 % 2) == 0 &&
      (reinterpret_cast<uintptr_t>(hi) % 4) == 0 && (reinterpret_cast<uintptr_t>(lo) % 4) == 0) {
    const int blocks = blocks_for_units((long long)rows1 * rows0 * ((ldo + kUnitCols2 - 1) / kUnitCols2));
    k_split_f32x2<<<blocks, 256, 0, s>>>(static_cast<const float *>(src), ld0, rows0, ld1, rows1, cols, ldo, ldo1,
                                         sign, absmax, scale_in, hi, lo, scale_out);
    return;
  }
  const int blocks = blocks_for_units((long long)rows1 * rows0 * ((ldo + kUnitCols - 1) / kUnitCols));
  if (f32)
    k_split_tensor<float><<<blocks, 256, 0, s>>>(static_cast<const float *>(src), ld0, rows0, ld1, rows1, ldc, cols,
                                                 ldo, ldo1, sign, absmax, scale_in, hi, lo, scale_out);
  else
    k_split_tensor<double><<<blocks, 256, 0, s>>>(static_cast<const double *>(src), ld0, rows0, ld1, rows1, ldc, cols,
                                                  ldo, ldo1, sign, absmax, scale_in, hi, lo, scale_out);
}

}  // namespace sox
