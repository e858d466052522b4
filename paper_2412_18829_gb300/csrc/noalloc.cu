// sox_sigma_fp64_noalloc: the FP64 bare-SOX chain with its scratch in a fixed
// device array, for callers that must not allocate device memory.
//
// Who needs this: code that runs where device allocation is off limits, e.g. a
// host process that hands all device memory to another runtime's fixed pool at
// start-up, or a caller that only has device pointers into someone else's
// buffers and may not grow the process's footprint.  Such callers cannot create
// a sox_handle (a handle allocates its workspace and status word with
// cudaMalloc).  This entry point takes no handle and calls no allocating
// routine; its intermediates live in kScratchBytes of static device memory that
// every GPU which loads the library holds until the process exits.
#include <algorithm>
#include <mutex>

#include <cuda.h>

#include "internal.h"

namespace {

// element counts rounded up to 32 doubles (256 bytes) so every slice stays aligned
inline size_t aligned(size_t count) { return (count + 31) & ~size_t(31); }

constexpr size_t kScratchBytes = SOX_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host code may not use g_scratch's name as a device address: it is a host-side
// stand-in.  The device address is looked up with the device current and cached
// per device together with the unique id of the context it was looked up under.
// A cudaDeviceReset (or any teardown of the primary context) gives the next
// context a new id, so the address is looked up again instead of reusing a
// stale one.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context, 0 when none is current yet.
int current_context_id(unsigned long long *id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || !f1 ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f2) {
      cudaGetLastError();
      return SOX_ERR_CUDA;
    }
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  *id = 0;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return SOX_ERR_CUDA;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return SOX_ERR_CUDA;
  return SOX_OK;
}

int scratch_address(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return SOX_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  int rc = current_context_id(&id);
  if (rc != SOX_OK) return rc;
  if (!g_addr[dev] || id == 0 || g_ctx_id[dev] != id) {
    // set-up for this device (first call, or a new context since the last one)
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SOX_ERR_CUDA;
    }
    rc = current_context_id(&id);   // the lookup has made the primary context current
    if (rc != SOX_OK) return rc;
    if (id == 0) return SOX_ERR_CUDA;
    g_addr[dev] = p;
    g_ctx_id[dev] = id;
  }
  *out = g_addr[dev];
  return SOX_OK;
}

// true when p is device (or managed) memory that belongs to device `dev`
bool on_device(const void *p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == dev;
  return a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int sox_sigma_fp64_noalloc(const sox_problem *p, const double *G, const double *X, const double *V,
                                      double *Sigma, void *stream) {
  if (!p || !G || !X || !V || !Sigma) return SOX_ERR_INVALID_ARG;
  if (p->n < 1 || p->n > SOX_MAX_N_AO || p->N < 1 || p->N > SOX_MAX_N_THC || p->n_tau < 2 ||
      p->n_tau > SOX_MAX_N_TAU || (p->n_spin != 1 && p->n_spin != 2))
    return SOX_ERR_SHAPE;
  if (p->nk[0] != 1 || p->nk[1] != 1 || p->nk[2] != 1 || p->dtype != SOX_REAL64) return SOX_ERR_UNSUPPORTED;
  if (!(p->beta > 0.0)) return SOX_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SOX_ERR_CUDA;
  }
  if (!on_device(G, dev) || !on_device(X, dev) || !on_device(V, dev) || !on_device(Sigma, dev))
    return SOX_ERR_INVALID_ARG;

  const int n = p->n, N = p->N, T = p->n_tau, S = p->n_spin;
  const size_t nn = (size_t)n * n, Nn2 = (size_t)N * nn;
  // scratch: mixed tensor [N][n][n], then per tau point of a chunk: A (or the
  // pair products while the mixed tensor is built) [n][N][n], G_Rq and G_wP^T
  // [N][n], D [N][N], T [N][n]; the chunk is as many tau points as fit.
  const size_t fixed = aligned(Nn2);
  const size_t per_tau = aligned(Nn2) + 3 * aligned((size_t)N * n) + aligned((size_t)N * N);
  if (fixed + per_tau > kScratchBytes / 8) return SOX_ERR_SHAPE;
  int c = (int)std::min<size_t>((kScratchBytes / 8 - fixed) / per_tau, (size_t)T);

  void *base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc != SOX_OK) return rc;
  double *w = static_cast<double *>(base);
  double *Um = w;
  double *big = Um + fixed;
  double *GR = big + (size_t)c * aligned(Nn2);
  double *GWt = GR + (size_t)c * aligned((size_t)N * n);
  double *Tm = GWt + (size_t)c * aligned((size_t)N * n);
  double *Dm = Tm + (size_t)c * aligned((size_t)N * n);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // A launch error left pending by the caller's earlier work on this thread is
  // cleared here, so the check after the launches below reports only this call's.
  cudaGetLastError();

  // Um[P][q][s] = sum_Q V[P][Q] X[Q][q] X[Q][s]
  sox::launch_pair_products_f64(X, big, N, n, s);
  sox::GemmF64 m;
  m.M = N; m.Nc = (int)nn; m.K = N;
  m.A = V; m.ai = N; m.ak = 1;
  m.B = big; m.bk = (long long)nn; m.bj = 1;
  m.C = Um; m.ci = (long long)nn; m.cj = 1;
  sox::launch_gemm_f64(m, s);
  for (int sp = 0; sp < S; ++sp) {
    const double *Gs = G + (long long)sp * T * nn;
    double *Ss = Sigma + (long long)sp * T * nn;
    for (int t0 = 0; t0 < T; t0 += c) {
      const int cc = std::min(c, T - t0);
      sox::GemmF64 g;  // G_Rq = X G
      g.M = N; g.Nc = n; g.K = n; g.batch = cc;
      g.A = X; g.ai = n; g.ak = 1;
      g.B = Gs + (long long)t0 * nn; g.sB = (long long)nn; g.bk = n; g.bj = 1;
      g.C = GR; g.sC = (long long)aligned((size_t)N * n); g.ci = n; g.cj = 1;
      sox::launch_gemm_f64(g, s);
      sox::GemmF64 gw = g;  // G_wP^T = X G^T
      gw.bk = 1; gw.bj = n;
      gw.C = GWt;
      sox::launch_gemm_f64(gw, s);
      sox::GemmF64 a;  // A[v][(P,q)] = -sum_s G(tau_{T-1-j})[s][v] Um[(P,q)][s]
      a.M = n; a.Nc = N * n; a.K = n; a.batch = cc;
      a.A = Gs + (long long)(T - 1 - t0) * nn; a.sA = -(long long)nn; a.ai = 1; a.ak = n;
      a.B = Um; a.bk = 1; a.bj = n;
      a.C = big; a.sC = (long long)aligned(Nn2); a.ci = (long long)N * n; a.cj = 1;
      a.alpha = -1.0;
      sox::launch_gemm_f64(a, s);
      sox::launch_sox_bcd_f64(big, (long long)aligned(Nn2), GR, (long long)aligned((size_t)N * n), GWt,
                              (long long)aligned((size_t)N * n), Um, Dm, (long long)aligned((size_t)N * N), n, N,
                              cc, s);
      sox::GemmF64 t;  // T[R][r] = sum_P D[P][R] X[P][r]
      t.M = N; t.Nc = n; t.K = N; t.batch = cc;
      t.A = Dm; t.sA = (long long)aligned((size_t)N * N); t.ai = 1; t.ak = N;
      t.B = X; t.bk = n; t.bj = 1;
      t.C = Tm; t.sC = (long long)aligned((size_t)N * n); t.ci = n; t.cj = 1;
      sox::launch_gemm_f64(t, s);
      sox::GemmF64 b;  // Sigma[t][r] = -sum_R X[R][t] T[R][r]
      b.M = n; b.Nc = n; b.K = N; b.batch = cc;
      b.A = X; b.ai = 1; b.ak = n;
      b.B = Tm; b.sB = (long long)aligned((size_t)N * n); b.bk = n; b.bj = 1;
      b.C = Ss + (long long)t0 * nn; b.sC = (long long)nn; b.ci = n; b.cj = 1;
      b.alpha = -1.0;
      sox::launch_gemm_f64(b, s);
    }
  }
  if (cudaGetLastError() != cudaSuccess) return SOX_ERR_CUDA;
  return SOX_OK;
}
