// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "smem_attr.h"
#include "thc_sox.h"

struct sox_context {
  int device = 0;
  int precision = SOX_PREC_FP64;
  long long spin_limit = 0;
  size_t ws_limit = 0;       // chunk budget override (sox_options.workspace_limit), 0 = defaults
  void *ws = nullptr;        // device workspace
  size_t ws_bytes = 0;
  void *aux = nullptr;       // second device buffer: partial results of composed entry points
  size_t aux_bytes = 0;
  int *d_status = nullptr;   // device status word for bounded waits
  int sm_count = 0;
  int v0 = 0, v1 = 0;        // sox_set_v_range: sums over the orbital index v run over [v0, v1) (v1 = 0: all)
  bool autotune = true;      // time the fused-kernel variants on the first call per shape
  int variant = 0;           // SOX_KERNEL_*: 0 = autotune, else the forced fused-kernel variant
  std::map<std::string, int> tuned;  // shape key -> chosen variant
  std::string last_error;
  // launch accounting (sox_profile_enable / sox_profile_read)
  bool prof = false;
  long long launches = 0;
  std::map<std::string, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> prof_events;
};

namespace sox {

// Counts `count` kernel launches; when profiling, brackets them with events.
struct ProfScope {
  sox_context *h;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  const char *name;
  ProfScope(sox_context *h_, const char *name_, cudaStream_t s_, int count = 1)
      : h(h_), s(s_), name(name_) {
    if (!h) return;
    h->launches += count;
    if (h->prof && name) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEventRecord(b, s);
      h->prof_events[name].push_back({a, b});
    }
  }
};

// Status carried through the host code; message goes to the handle.
struct Status {
  int code = SOX_OK;
  std::string msg;
  static Status ok() { return {}; }
  bool good() const { return code == SOX_OK; }
};

#define SOX_CUDA_TRY(expr)                                                          \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ::sox::Status{SOX_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define SOX_TRY(expr)                 \
  do {                                \
    ::sox::Status s_ = (expr);        \
    if (!s_.good()) return s_;        \
  } while (0)

// The handle's v range clamped to [0, n]: *lo <= *hi.
inline void v_range(const sox_context *h, int n, int *lo, int *hi) {
  int b = (h && h->v1 > 0) ? (h->v1 < n ? h->v1 : n) : n;
  int a = h ? h->v0 : 0;
  a = a < 0 ? 0 : (a > b ? b : a);
  *lo = a;
  *hi = b;
}
inline bool v_range_is_full(const sox_context *h, int n) {
  int a, b;
  v_range(h, n, &a, &b);
  return a == 0 && b == n;
}

// Bump allocator over the handle workspace (256-byte aligned slices).
// Chunk budget of a planner: the handle's override, else the planner's default.
inline size_t chunk_budget(const sox_context *h, size_t dflt) { return (h && h->ws_limit) ? h->ws_limit : dflt; }

struct Arena {
  char *base = nullptr;
  size_t cap = 0, off = 0;
  template <class T>
  T *take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    T *p = reinterpret_cast<T *>(base + off);
    off += bytes;
    return off <= cap ? p : nullptr;
  }
};
inline size_t aligned_bytes(size_t count, size_t elem) { return (count * elem + 255) & ~size_t(255); }

// ---------------- FP64 CUDA-core kernels (fp64_kernels.cu) ----------------
// Strided batched GEMM: C[b](i,j) = alpha * sum_k A[b](i,k) B[b](k,j) + beta * C[b](i,j)
// Element (i,k) of A at A + b*sA + i*ai + k*ak, and likewise for B and C.
struct GemmF64 {
  int M = 0, Nc = 0, K = 0, batch = 1;
  const double *A = nullptr; long long sA = 0, ai = 0, ak = 0;
  const double *B = nullptr; long long sB = 0, bk = 0, bj = 0;
  double *C = nullptr; long long sC = 0, ci = 0, cj = 0;
  double alpha = 1.0, beta = 0.0;
  const int *skip = nullptr;  // optional per-batch flags: batch b is not computed when skip[b] != 0
};
void launch_gemm_f64(const GemmF64 &g, cudaStream_t s);

// Y[Q][q][s] = X[Q][q] * X[Q][s]   (pair products feeding the mixed THC tensor)
void launch_pair_products_f64(const double *X, double *Y, int N, int n, cudaStream_t s);

// D[b][P][R] = sum_v (sum_q A[b][v][P][q] GR[b][R][q]) * (sum_w GWt[b][P][w] U2[R][v][w])
// b runs over `batch` (tau points of one spin); strides in elements.  The v sum runs over
// [v0, v1) (v1 <= 0: all n).
void launch_sox_bcd_f64(const double *A, long long sA, const double *GR, long long sGR,
                        const double *GWt, long long sGW, const double *U2, double *D,
                        long long sD, int n, int N, int batch, cudaStream_t s, int v0 = 0, int v1 = 0);

// phi_part[b] = sum_tr Sigma[b][t][r] * Gm[b][r][t] with Gm[b] = -G[n_tau-1-tau(b)]
void launch_trace_sigma_gminus(const double *Sigma, const double *G, int n, int n_tau,
                               int n_blocks_spin, double *partial, cudaStream_t s);
// phi[s] = 1/4 sum_j w[j] partial[s][j]  (sequential order, deterministic)
void launch_phi_finish(const double *partial, const double *w, int n_tau, int n_spin,
                       double *phi, cudaStream_t s);

// dG[s][j][r][t] = -dphi[s] * w[j] * Sigma[s][n_tau-1-j][t][r]
void launch_dG_from_sigma(const double *Sigma, const double *w, const double *dphi, int n,
                          int n_tau, int n_spin, double *dG, cudaStream_t s);

// Pi[P][Q] = - sum_j w[j] GPQ[j][P][Q] * GPQ[n_tau-1-j][Q][P]
void launch_pi0_reduce(const double *GPQ, const double *w, int N, int n_tau, double *Pi,
                       cudaStream_t s);

// Gauss-Jordan on the augmented [K | Bm] (N x 2N, row-major, in place):
// returns the solution K^-1 Bm in the right half.  piv_info: device int[2].
void launch_gj_step(double *Aug, int N, int k, int *piv_info, cudaStream_t s);
void launch_build_gj_system(const double *V, const double *Pi, double *Aug, int N, cudaStream_t s);
void launch_copy_right_half(const double *Aug, double *W, int N, cudaStream_t s);
// dst[i] = a[i] + b[i]
void launch_add_f64(const double *a, const double *b, double *dst, long long count, cudaStream_t s);
// flag[b] = 1 when G[b] (n x n) equals its transpose to 1e-14 of max|G[b]|, else 0
void launch_symmetry_flags(const double *G, int n, int batch, int *flag, cudaStream_t s);
void launch_neg_reflect(const double *src, double *dst, long long mat, int n_tau, int count,
                        cudaStream_t s);

}  // namespace sox
