// C-ABI entry points: handle lifecycle, argument validation, host/device
// staging, and the orchestration of the THC-SOX chain (Sec. II C) on one stream.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "adjoint.h"
#include "dynamic.h"
#include "internal.h"
#include "ctc.h"
#include "kpoint.h"
#include "scloop.h"
#include "tc_path.h"

using sox::Arena;
using sox::GemmF64;
using sox::Status;

namespace {

constexpr size_t kDefaultBudget = size_t(12) << 30;  // τ-chunking budget for intermediates

Status validate(const sox_problem *p, bool need_molecule = true) {
  if (!p) return {SOX_ERR_INVALID_ARG, "problem descriptor is NULL"};
  if (p->n < 1 || p->n > SOX_MAX_N_AO) return {SOX_ERR_SHAPE, "n out of range [1, SOX_MAX_N_AO]"};
  if (p->N < 1 || p->N > SOX_MAX_N_THC) return {SOX_ERR_SHAPE, "N out of range [1, SOX_MAX_N_THC]"};
  if (p->n_tau < 2 || p->n_tau > SOX_MAX_N_TAU) return {SOX_ERR_SHAPE, "n_tau out of range [2, SOX_MAX_N_TAU]"};
  if (p->n_spin != 1 && p->n_spin != 2) return {SOX_ERR_SHAPE, "n_spin must be 1 or 2"};
  for (int d = 0; d < 3; ++d)
    if (p->nk[d] < 1 || p->nk[d] > 64) return {SOX_ERR_SHAPE, "k-mesh entries must be in [1, 64]"};
  if (p->dtype != SOX_REAL64 && p->dtype != SOX_COMPLEX128) return {SOX_ERR_INVALID_ARG, "unknown dtype"};
  if (!(p->beta > 0.0) || !std::isfinite(p->beta)) return {SOX_ERR_INVALID_ARG, "beta must be finite and > 0"};
  if (need_molecule) {
    if (p->nk[0] * p->nk[1] * p->nk[2] != 1)
      return {SOX_ERR_UNSUPPORTED, "k-point meshes (solids) are not implemented by this entry point"};
    if (p->dtype != SOX_REAL64)
      return {SOX_ERR_UNSUPPORTED, "complex data are not implemented by this entry point"};
  }
  return Status::ok();
}

int finish(sox_handle h, const Status &s) {
  if (h) h->last_error = s.good() ? std::string() : s.msg;
  return s.code;
}

// Whether a pointer is device-accessible (device or managed memory).
Status is_device_ptr(const void *ptr, bool *dev) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *dev = false;
    return Status::ok();
  }
  *dev = (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
  return Status::ok();
}

struct Staged {
  // inputs: device pointer to use; outputs: device pointer to write + host target
  const double *in = nullptr;
  double *out = nullptr;
  double *host_out = nullptr;
  size_t count = 0;
  bool host = false;
};

class Call {
 public:
  Call(sox_handle h, void *stream) : h_(h), s_(reinterpret_cast<cudaStream_t>(stream)) {}
  cudaStream_t stream() const { return s_; }

  // Register an input (may be NULL when optional); returns where the kernels read it.
  Status input(const double *p, size_t count, Staged *st) {
    st->count = count;
    if (!p) return Status::ok();
    bool dev = false;
    SOX_TRY(is_device_ptr(p, &dev));
    st->host = !dev;
    st->in = p;
    if (st->host) staged_in_.push_back(st), stage_bytes_ += sox::aligned_bytes(count, 8);
    return Status::ok();
  }
  Status output(double *p, size_t count, Staged *st) {
    st->count = count;
    if (!p) return Status::ok();
    bool dev = false;
    SOX_TRY(is_device_ptr(p, &dev));
    st->host = !dev;
    st->out = p;
    if (st->host) {
      st->host_out = p;
      staged_out_.push_back(st);
      stage_bytes_ += sox::aligned_bytes(count, 8);
    }
    return Status::ok();
  }

  // Ensure workspace >= compute_bytes + staging, then copy host inputs in.
  Status begin(size_t compute_bytes, Arena *arena) {
    size_t need = compute_bytes + stage_bytes_ + 4096;
    if (need > h_->ws_bytes) {
      if (h_->ws) {
        SOX_CUDA_TRY(cudaDeviceSynchronize());
        SOX_CUDA_TRY(cudaFree(h_->ws));
        h_->ws = nullptr;
        h_->ws_bytes = 0;
      }
      if (cudaMalloc(&h_->ws, need) != cudaSuccess) {
        cudaGetLastError();
        return {SOX_ERR_OOM, "workspace allocation of " + std::to_string(need) + " bytes failed"};
      }
      h_->ws_bytes = need;
    }
    arena->base = static_cast<char *>(h_->ws);
    arena->cap = h_->ws_bytes;
    arena->off = 0;
    for (Staged *st : staged_in_) {
      double *d = arena->take<double>(st->count);
      SOX_CUDA_TRY(cudaMemcpyAsync(d, st->in, st->count * 8, cudaMemcpyHostToDevice, s_));
      st->in = d;
    }
    for (Staged *st : staged_out_) st->out = arena->take<double>(st->count);
    return Status::ok();
  }

  Status end() {
    for (Staged *st : staged_out_)
      SOX_CUDA_TRY(cudaMemcpyAsync(st->host_out, st->out, st->count * 8, cudaMemcpyDeviceToHost, s_));
    if (!staged_out_.empty()) SOX_CUDA_TRY(cudaStreamSynchronize(s_));
    SOX_CUDA_TRY(cudaGetLastError());
    return Status::ok();
  }

 private:
  sox_handle h_;
  cudaStream_t s_;
  std::vector<Staged *> staged_in_, staged_out_;
  size_t stage_bytes_ = 0;
};

Status bind_device(sox_handle h) {
  int cur = -1;
  SOX_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != h->device) SOX_CUDA_TRY(cudaSetDevice(h->device));
  return Status::ok();
}

// --------------------------- FP64 orchestration ---------------------------

struct Dims {
  int n, N, T, S;
  long long nn() const { return (long long)n * n; }
};

// Projections for cc tau points starting at t0 of one spin block (FP64).
void project_chunk(sox_handle H, const double *Gs, const double *X, const Dims &d, int t0, int cc,
                   double *GR, double *GWt, cudaStream_t s) {
  GemmF64 g;  // GR[b][R][q] = sum_u X[R][u] G[t0+b][u][q]
  g.M = d.N; g.Nc = d.n; g.K = d.n; g.batch = cc;
  g.A = X; g.ai = d.n; g.ak = 1;
  g.B = Gs + (long long)t0 * d.nn(); g.sB = d.nn(); g.bk = d.n; g.bj = 1;
  g.C = GR; g.sC = (long long)d.N * d.n; g.ci = d.n; g.cj = 1;
  GemmF64 h = g;  // GWt[b][P][w] = sum_p X[P][p] G[t0+b][w][p]
  h.bk = 1; h.bj = d.n;
  h.C = GWt;
  sox::ProfScope ps(H, "project_f64", s, 2);
  sox::launch_gemm_f64(g, s);
  sox::launch_gemm_f64(h, s);
}

// Um[P][q][s] = sum_Q U[P][Q] X[Q][q] X[Q][s]   (Eq. U_contraction at k = 0)
void mixed_tensor_f64(sox_handle H, const double *U, const double *X, const Dims &d, double *Y,
                      double *Um, cudaStream_t s) {
  GemmF64 g;
  g.M = d.N; g.Nc = (int)d.nn(); g.K = d.N;
  g.A = U; g.ai = d.N; g.ak = 1;
  g.B = Y; g.bk = d.nn(); g.bj = 1;
  g.C = Um; g.ci = d.nn(); g.cj = 1;
  sox::ProfScope ps(H, "mixed_f64", s, 2);
  sox::launch_pair_products_f64(X, Y, d.N, d.n, s);
  sox::launch_gemm_f64(g, s);
}

int tau_chunk(sox_handle h, const Dims &d, size_t per_tau_bytes, size_t fixed_bytes) {
  const size_t total = sox::chunk_budget(h, kDefaultBudget);
  size_t budget = total > fixed_bytes ? total - fixed_bytes : 0;
  long long c = per_tau_bytes ? (long long)(budget / per_tau_bytes) : d.T;
  if (c < 1) c = 1;
  if (c > d.T) c = d.T;
  return (int)c;
}

size_t sigma_fp64_bytes(sox_handle h, const Dims &d, bool two_slots, int *chunk) {
  size_t Nn2 = (size_t)d.N * d.nn();
  size_t fixed = sox::aligned_bytes(Nn2, 8) * (two_slots ? 2 : 1);
  size_t per_tau = 8 * (Nn2 + 3 * (size_t)d.N * d.n + (size_t)d.N * d.N) + 1024;
  int c = tau_chunk(h, d, per_tau, fixed);
  if (chunk) *chunk = c;
  return fixed + sox::aligned_bytes(std::max<size_t>(Nn2 * c, Nn2), 8) +
         4 * sox::aligned_bytes((size_t)c * d.N * std::max(d.n, d.N), 8);
}

// Sigma for every spin and tau point; U1 == U2 allowed (bare SOX).
Status sigma_fp64(sox_handle H, const Dims &d, const double *G, const double *X, const double *U1,
                  const double *U2, double *Sigma, Arena &ar, cudaStream_t s) {
  const bool two = (U1 != U2);
  int c = 1;
  sigma_fp64_bytes(H, d, two, &c);
  const size_t Nn2 = (size_t)d.N * d.nn();
  double *Um1 = ar.take<double>(Nn2);
  double *Um2 = two ? ar.take<double>(Nn2) : Um1;
  double *big = ar.take<double>(std::max<size_t>(Nn2 * c, Nn2));
  double *GR = ar.take<double>((size_t)c * d.N * d.n);
  double *GWt = ar.take<double>((size_t)c * d.N * d.n);
  double *Dm = ar.take<double>((size_t)c * d.N * d.N);
  double *Tm = ar.take<double>((size_t)c * d.N * d.n);
  if (!Tm) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  mixed_tensor_f64(H, U1, X, d, big, Um1, s);
  if (two) mixed_tensor_f64(H, U2, X, d, big, Um2, s);
  for (int sp = 0; sp < d.S; ++sp) {
    const double *Gs = G + (long long)sp * d.T * d.nn();
    double *Ss = Sigma + (long long)sp * d.T * d.nn();
    for (int t0 = 0; t0 < d.T; t0 += c) {
      int cc = std::min(c, d.T - t0);
      project_chunk(H, Gs, X, d, t0, cc, GR, GWt, s);
      // A[b][v][(P,q)] = sum_s G(-tau)[s][v] Um1[(P,q)][s],  G(-tau_j) = -G(tau_{T-1-j})
      GemmF64 a;
      a.M = d.n; a.Nc = d.N * d.n; a.K = d.n; a.batch = cc;
      a.A = Gs + (long long)(d.T - 1 - t0) * d.nn(); a.sA = -d.nn(); a.ai = 1; a.ak = d.n;
      a.B = Um1; a.bk = 1; a.bj = d.n;
      a.C = big; a.sC = (long long)Nn2; a.ci = (long long)d.N * d.n; a.cj = 1;
      a.alpha = -1.0;
      {
        sox::ProfScope ps(H, "A_f64", s);
        sox::launch_gemm_f64(a, s);
      }
      {  // D[b][P][R] = sum_v B o C
        sox::ProfScope ps(H, "sox_bcd", s);
        sox::launch_sox_bcd_f64(big, (long long)Nn2, GR, (long long)d.N * d.n, GWt,
                                (long long)d.N * d.n, Um2, Dm, (long long)d.N * d.N, d.n, d.N, cc, s,
                                H ? H->v0 : 0, H ? H->v1 : 0);
      }
      // T[b][R][r] = sum_P D[b][P][R] X[P][r]
      GemmF64 t;
      t.M = d.N; t.Nc = d.n; t.K = d.N; t.batch = cc;
      t.A = Dm; t.sA = (long long)d.N * d.N; t.ai = 1; t.ak = d.N;
      t.B = X; t.bk = d.n; t.bj = 1;
      t.C = Tm; t.sC = (long long)d.N * d.n; t.ci = d.n; t.cj = 1;
      // Sigma[t][r] = -sum_R X[R][t] T[R][r]
      GemmF64 b;
      b.M = d.n; b.Nc = d.n; b.K = d.N; b.batch = cc;
      b.A = X; b.ai = 1; b.ak = d.n;
      b.B = Tm; b.sB = (long long)d.N * d.n; b.bk = d.n; b.bj = 1;
      b.C = Ss + (long long)t0 * d.nn(); b.sC = d.nn(); b.ci = d.n; b.cj = 1;
      b.alpha = -1.0;
      {
        sox::ProfScope ps(H, "backproject_f64", s, 2);
        sox::launch_gemm_f64(t, s);
        sox::launch_gemm_f64(b, s);
      }
    }
  }
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

Dims dims_of(const sox_problem *p) { return Dims{p->n, p->N, p->n_tau, p->n_spin}; }

size_t sigma_bytes(sox_handle h, const Dims &d, bool two) {
  if (h->precision == SOX_PREC_F16X2) return sox::tc_sigma_bytes(h, d.n, d.N, d.T, d.S, two);
  return sigma_fp64_bytes(h, d, two, nullptr);
}

Status sigma_any(sox_handle h, const Dims &d, const double *G, const double *X, const double *U1,
                 const double *U2, double *Sigma, Arena &ar, cudaStream_t s) {
  if (h->precision == SOX_PREC_F16X2)
    return sox::tc_sigma(h, d.n, d.N, d.T, d.S, G, X, U1, U2, Sigma, ar, s);
  return sigma_fp64(h, d, G, X, U1, U2, Sigma, ar, s);
}

// Solids (complex data, any k-mesh): the momentum-resolved chain in FP64 complex.
Status run_sigma_complex(sox_handle h, const sox_problem *p, const double *G, const double *X,
                         const double *U1, const double *U2, double *Sigma, void *stream) {
  SOX_TRY(validate(p, false));
  if (p->dtype != SOX_COMPLEX128)
    return {SOX_ERR_UNSUPPORTED, "k-point meshes need complex data (SOX_COMPLEX128)"};
  SOX_TRY(bind_device(h));
  const int nk = p->nk[0] * p->nk[1] * p->nk[2];
  const size_t nn = (size_t)p->n * p->n;
  Call call(h, stream);
  Staged sG, sX, s1, s2, sS;
  SOX_TRY(call.input(G, 2 * (size_t)p->n_spin * nk * p->n_tau * nn, &sG));
  SOX_TRY(call.input(X, 2 * (size_t)nk * p->N * p->n, &sX));
  SOX_TRY(call.input(U1, 2 * (size_t)nk * p->N * p->N, &s1));
  const bool same = (U1 == U2);
  if (!same) SOX_TRY(call.input(U2, 2 * (size_t)nk * p->N * p->N, &s2));
  SOX_TRY(call.output(Sigma, 2 * (size_t)p->n_spin * nk * p->n_tau * nn, &sS));
  Arena ar;
  if (h->precision == SOX_PREC_F16X2) {
    SOX_TRY(call.begin(sox::kpoint_tc_bytes(h, p, !same), &ar));
    SOX_TRY(sox::kpoint_sigma_tc(h, p, sG.in, sX.in, s1.in, same ? s1.in : s2.in, sS.out, ar, call.stream()));
    return call.end();
  }
  const sox::KpointPlan pl = sox::kpoint_plan(h, p->n, p->N, p->n_tau, p->n_spin, p->nk);
  SOX_TRY(call.begin(pl.bytes + (same ? 0 : 16 * (size_t)nk * nk * p->N * nn), &ar));
  SOX_TRY(sox::kpoint_sigma_f64(h, p, sG.in, sX.in, s1.in, same ? s1.in : s2.in, sS.out, ar, call.stream()));
  return call.end();
}

Status run_sigma(sox_handle h, const sox_problem *p, const double *G, const double *X,
                 const double *U1, const double *U2, double *Sigma, void *stream) {
  if (!h) return {SOX_ERR_INVALID_ARG, "handle is NULL"};
  if (!G || !X || !U1 || !U2 || !Sigma) return {SOX_ERR_INVALID_ARG, "a required tensor pointer is NULL"};
  if (p && (p->dtype == SOX_COMPLEX128 || p->nk[0] * p->nk[1] * p->nk[2] != 1))
    return run_sigma_complex(h, p, G, X, U1, U2, Sigma, stream);
  SOX_TRY(validate(p));
  SOX_TRY(bind_device(h));
  const Dims d = dims_of(p);
  Call call(h, stream);
  Staged sG, sX, s1, s2, sS;
  SOX_TRY(call.input(G, (size_t)d.S * d.T * d.nn(), &sG));
  SOX_TRY(call.input(X, (size_t)d.N * d.n, &sX));
  SOX_TRY(call.input(U1, (size_t)d.N * d.N, &s1));
  const bool same = (U1 == U2);
  if (!same) SOX_TRY(call.input(U2, (size_t)d.N * d.N, &s2));
  SOX_TRY(call.output(Sigma, (size_t)d.S * d.T * d.nn(), &sS));
  Arena ar;
  SOX_TRY(call.begin(sigma_bytes(h, d, !same), &ar));
  const double *u2 = same ? s1.in : s2.in;
  SOX_TRY(sigma_any(h, d, sG.in, sX.in, s1.in, u2, sS.out, ar, call.stream()));
  return call.end();
}

// dst = a - b
__global__ void k_sub_f64(const double *a, const double *b, double *dst, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = a[e] - b[e];
}

// Grows the handle's second buffer (synchronises the device when it reallocates).
Status ensure_aux(sox_handle h, size_t bytes) {
  if (bytes <= h->aux_bytes) return Status::ok();
  if (h->aux) {
    SOX_CUDA_TRY(cudaDeviceSynchronize());
    SOX_CUDA_TRY(cudaFree(h->aux));
    h->aux = nullptr;
    h->aux_bytes = 0;
  }
  if (cudaMalloc(&h->aux, bytes) != cudaSuccess) {
    cudaGetLastError();
    return {SOX_ERR_OOM, "allocation of " + std::to_string(bytes) + " bytes for partial results failed"};
  }
  h->aux_bytes = bytes;
  return Status::ok();
}

}  // namespace

// ================================ C ABI ===================================
extern "C" {

int sox_version(void) { return 100; }

int sox_create(sox_handle *out, const sox_options *opt) {
  if (!out) return SOX_ERR_INVALID_ARG;
  *out = nullptr;
  sox_options o{SOX_PREC_FP64, 0, 0, 0, 0};
  if (opt) o = *opt;
  if (o.precision != SOX_PREC_FP64 && o.precision != SOX_PREC_F16X2) return SOX_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return SOX_ERR_CUDA;
  }
  if (o.device < 0 || o.device >= ndev) return SOX_ERR_INVALID_ARG;
  sox_context *h = new (std::nothrow) sox_context();
  if (!h) return SOX_ERR_OOM;
  h->device = o.device;
  h->precision = o.precision;
  h->spin_limit = o.spin_limit > 0 ? o.spin_limit : (1LL << 22);
  if (o.workspace_limit < 0) {
    delete h;
    return SOX_ERR_INVALID_ARG;
  }
  h->ws_limit = (size_t)o.workspace_limit;
  h->autotune = (o.no_autotune == 0);
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(o.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, o.device) != cudaSuccess ||
      cudaMalloc(&h->d_status, 64) != cudaSuccess || cudaMemset(h->d_status, 0, 64) != cudaSuccess) {
    cudaGetLastError();
    if (h->d_status) cudaFree(h->d_status);
    delete h;
    return SOX_ERR_CUDA;
  }
  if (prev >= 0 && prev != o.device) cudaSetDevice(prev);
  *out = h;
  return SOX_OK;
}

int sox_destroy(sox_handle h) {
  if (!h) return SOX_ERR_INVALID_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  sox::tc_release(h);
  sox_profile_enable(h, 0);
  if (h->ws) cudaFree(h->ws);
  if (h->aux) cudaFree(h->aux);
  if (h->d_status) cudaFree(h->d_status);
  if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
  delete h;
  return SOX_OK;
}

int sox_profile_enable(sox_handle h, int enable) {
  if (!h) return SOX_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  for (auto &kv : h->prof_events)
    for (auto &e : kv.second) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  h->prof_events.clear();
  h->launches = 0;
  h->prof = enable != 0;
  return SOX_OK;
}

int sox_profile_read(sox_handle h, const char *kernel, long long *launches, double *ms) {
  if (!h || !launches || !ms) return SOX_ERR_INVALID_ARG;
  *launches = 0;
  *ms = 0.0;
  if (!kernel) {
    *launches = h->launches;
    return SOX_OK;
  }
  cudaSetDevice(h->device);
  if (cudaDeviceSynchronize() != cudaSuccess) return finish(h, {SOX_ERR_CUDA, "device sync failed"});
  auto it = h->prof_events.find(kernel);
  if (it == h->prof_events.end()) return SOX_OK;
  double tot = 0.0;
  for (auto &e : it->second) {
    float f = 0.f;
    if (cudaEventElapsedTime(&f, e.first, e.second) != cudaSuccess) {
      cudaGetLastError();
      return finish(h, {SOX_ERR_CUDA, "cudaEventElapsedTime failed"});
    }
    tot += f;
  }
  *launches = (long long)it->second.size();
  *ms = tot;
  return SOX_OK;
}

int sox_check_device(sox_handle h) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(bind_device(h));
    SOX_CUDA_TRY(cudaDeviceSynchronize());
    int word = 0;
    SOX_CUDA_TRY(cudaMemcpy(&word, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (word) {
      SOX_CUDA_TRY(cudaMemset(h->d_status, 0, sizeof(int)));
      return {SOX_ERR_TIMEOUT, "a device-side wait reached its iteration cap (status word " +
                                   std::to_string(word) + "); the affected results are invalid"};
    }
    return Status::ok();
  }();
  return finish(h, st);
}

const char *sox_last_error(sox_handle h) { return h ? h->last_error.c_str() : "handle is NULL"; }

int sox_set_v_range(sox_handle h, int v0, int v1) {
  if (!h) return SOX_ERR_INVALID_ARG;
  if (v0 < 0 || (v1 > 0 && v1 < v0)) return finish(h, {SOX_ERR_INVALID_ARG, "v range must satisfy 0 <= v0 <= v1"});
  h->v0 = v0;
  h->v1 = v1;
  return finish(h, Status::ok());
}

int sox_set_kernel_variant(sox_handle h, int variant) {
  if (!h) return SOX_ERR_INVALID_ARG;
  if (variant < SOX_KERNEL_AUTO || variant > SOX_KERNEL_PAIR)
    return finish(h, {SOX_ERR_INVALID_ARG, "unknown fused-kernel variant"});
  h->variant = variant;
  return finish(h, Status::ok());
}

int sox_reserve(sox_handle h, const sox_problem *p) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = validate(p);
  if (st.good()) st = bind_device(h);
  if (st.good()) {
    const Dims d = dims_of(p);
    size_t need = sigma_bytes(h, d, true);
    size_t io = 8 * ((size_t)2 * d.S * d.T * d.nn() + (size_t)d.N * d.n + 2 * (size_t)d.N * d.N);
    Call call(h, nullptr);
    Arena ar;
    st = call.begin(need + io, &ar);
  }
  return finish(h, st);
}

int sox_tau_grid(int n_tau, double beta, double *tau, double *w) {
  if (n_tau < 2 || n_tau > SOX_MAX_N_TAU || !(beta > 0.0) || !tau || !w) return SOX_ERR_INVALID_ARG;
  const int M = n_tau - 1;
  const double pi = 3.14159265358979323846;
  for (int j = 0; j < n_tau; ++j) tau[j] = 0.5 * beta * (1.0 - std::cos(pi * j / M));
  tau[0] = 0.0;
  tau[M] = beta;
  for (int j = 0; j < n_tau / 2; ++j) tau[M - j] = beta - tau[j];
  if (n_tau % 2) tau[M / 2] = 0.5 * beta;
  // Clenshaw-Curtis weights on [-1, 1] (cosine-series form), scaled by beta/2
  for (int j = 0; j < n_tau; ++j) {
    double s = 1.0;
    for (int k = 1; k <= M / 2; ++k) {
      double b = (2 * k == M) ? 1.0 : 2.0;
      s -= b * std::cos(2.0 * pi * (double)j * k / M) / (4.0 * k * k - 1.0);
    }
    double c = (j == 0 || j == M) ? 1.0 : 2.0;
    w[j] = 0.5 * beta * c * s / M;
  }
  for (int j = 0; j < n_tau / 2; ++j) {
    double a = 0.5 * (w[j] + w[M - j]);
    w[j] = w[M - j] = a;
  }
  return SOX_OK;
}

int thc_project_G(sox_handle h, const sox_problem *p, const double *G, const double *X,
                  double *G_Rq, double *G_wP, double *G_PQ, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(validate(p));
    if (!G || !X || (!G_Rq && !G_wP && !G_PQ)) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const Dims d = dims_of(p);
    const size_t nb = (size_t)d.S * d.T;
    Call call(h, stream);
    Staged sG, sX, oR, oW, oP;
    SOX_TRY(call.input(G, nb * d.nn(), &sG));
    SOX_TRY(call.input(X, (size_t)d.N * d.n, &sX));
    SOX_TRY(call.output(G_Rq, nb * d.N * d.n, &oR));
    SOX_TRY(call.output(G_wP, nb * d.N * d.n, &oW));
    SOX_TRY(call.output(G_PQ, nb * d.N * d.N, &oP));
    Arena ar;
    SOX_TRY(call.begin(G_PQ && !G_Rq ? sox::aligned_bytes(nb * d.N * d.n, 8) : 0, &ar));
    double *gr = oR.out ? oR.out : (G_PQ ? ar.take<double>(nb * d.N * d.n) : nullptr);
    cudaStream_t s = call.stream();
    GemmF64 g;  // GR[b][R][q] = sum_u X[R][u] G[b][u][q]
    g.M = d.N; g.Nc = d.n; g.K = d.n; g.batch = (int)nb;
    g.A = sX.in; g.ai = d.n; g.ak = 1;
    g.B = sG.in; g.sB = d.nn(); g.bk = d.n; g.bj = 1;
    g.C = gr; g.sC = (long long)d.N * d.n; g.ci = d.n; g.cj = 1;
    sox::ProfScope ps(h, "project_f64", s, (gr ? 1 : 0) + (oW.out ? 1 : 0) + (oP.out ? 1 : 0));
    if (gr) sox::launch_gemm_f64(g, s);
    if (oW.out) {  // G_wP[b][w][P] = sum_p G[b][w][p] X[P][p]
      GemmF64 w;
      w.M = d.n; w.Nc = d.N; w.K = d.n; w.batch = (int)nb;
      w.A = sG.in; w.sA = d.nn(); w.ai = d.n; w.ak = 1;
      w.B = sX.in; w.bk = 1; w.bj = d.n;
      w.C = oW.out; w.sC = (long long)d.N * d.n; w.ci = d.N; w.cj = 1;
      sox::launch_gemm_f64(w, s);
    }
    if (oP.out) {  // G_PQ[b][P][Q] = sum_q GR[b][P][q] X[Q][q]
      GemmF64 q;
      q.M = d.N; q.Nc = d.N; q.K = d.n; q.batch = (int)nb;
      q.A = gr; q.sA = (long long)d.N * d.n; q.ai = d.n; q.ak = 1;
      q.B = sX.in; q.bk = 1; q.bj = d.n;
      q.C = oP.out; q.sC = (long long)d.N * d.N; q.ci = d.N; q.cj = 1;
      sox::launch_gemm_f64(q, s);
    }
    return call.end();
  }();
  return finish(h, st);
}

int sox_sigma(sox_handle h, const sox_problem *p, const double *G, const double *X,
              const double *V, double *Sigma, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  return finish(h, run_sigma(h, p, G, X, V, V, Sigma, stream));
}

int sox_sigma_general(sox_handle h, const sox_problem *p, const double *G, const double *X,
                      const double *U1, const double *U2, double *Sigma, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  return finish(h, run_sigma(h, p, G, X, U1, U2, Sigma, stream));
}

int sosex_static_sigma(sox_handle h, const sox_problem *p, const double *G, const double *X,
                       const double *V, const double *W0, int slot, double *Sigma,
                       void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  if (slot != 1 && slot != 2) return finish(h, {SOX_ERR_INVALID_ARG, "slot must be 1 or 2"});
  if (V == W0 && V) return finish(h, {SOX_ERR_INVALID_ARG, "V and W0 must be distinct buffers"});
  const double *u1 = slot == 1 ? W0 : V, *u2 = slot == 1 ? V : W0;
  return finish(h, run_sigma(h, p, G, X, u1, u2, Sigma, stream));
}

int g3w2_static_sigma(sox_handle h, const sox_problem *p, const double *G, const double *X, const double *W0,
                      double *Sigma, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  return finish(h, run_sigma(h, p, G, X, W0, W0, Sigma, stream));
}

int sosex2_static_sigma(sox_handle h, const sox_problem *p, const double *G, const double *X, const double *V,
                        const double *W0, double *Sigma, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    if (!p) return {SOX_ERR_INVALID_ARG, "problem descriptor is NULL"};
    SOX_TRY(validate(p, false));
    if (!G || !X || !V || !W0 || !Sigma) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    if (V == W0) return {SOX_ERR_INVALID_ARG, "V and W0 must be distinct buffers"};
    SOX_TRY(bind_device(h));
    const long long mult = p->dtype == SOX_COMPLEX128 ? 2 : 1;
    const long long nk = (long long)p->nk[0] * p->nk[1] * p->nk[2];
    const long long nsig = mult * p->n_spin * nk * p->n_tau * (long long)p->n * p->n;
    const long long nX = mult * nk * (long long)p->N * p->n;
    const long long nV = mult * nk * (long long)p->N * p->N;
    // host tensors are staged through the second buffer: [part][W_d][G][X][V][W0][Sigma]
    const void *ptrs[5] = {G, X, V, W0, Sigma};
    const long long cnt[5] = {nsig, nX, nV, nV, nsig};
    bool host[5];
    for (int i = 0; i < 5; ++i) {
      cudaPointerAttributes a{};
      if (cudaPointerGetAttributes(&a, ptrs[i]) != cudaSuccess) {
        cudaGetLastError();
        a.type = cudaMemoryTypeUnregistered;
      }
      host[i] = (a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered);
      if (!host[i] && a.device != h->device)
        return {SOX_ERR_INVALID_ARG, "device tensors must live on the handle's GPU"};
    }
    size_t need = sox::aligned_bytes(nsig, 8) + sox::aligned_bytes(nV, 8);
    for (int i = 0; i < 5; ++i)
      if (host[i]) need += sox::aligned_bytes(cnt[i], 8);
    SOX_TRY(ensure_aux(h, need));
    char *base = static_cast<char *>(h->aux);
    double *part = reinterpret_cast<double *>(base);
    double *Wd = reinterpret_cast<double *>(base + sox::aligned_bytes(nsig, 8));
    size_t off = sox::aligned_bytes(nsig, 8) + sox::aligned_bytes(nV, 8);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *dev[5];
    for (int i = 0; i < 5; ++i) {
      if (!host[i]) {
        dev[i] = const_cast<double *>(static_cast<const double *>(ptrs[i]));
        continue;
      }
      dev[i] = reinterpret_cast<double *>(base + off);
      off += sox::aligned_bytes(cnt[i], 8);
      if (i < 4) SOX_CUDA_TRY(cudaMemcpyAsync(dev[i], ptrs[i], 8 * (size_t)cnt[i], cudaMemcpyHostToDevice, s));
    }
    const int grid = (int)std::max<long long>(1, std::min<long long>((nV + 255) / 256, 65535 * 8));
    k_sub_f64<<<grid, 256, 0, s>>>(dev[3], dev[2], Wd, nV);     // W_d = W0 - v
    ++h->launches;
    SOX_CUDA_TRY(cudaGetLastError());
    SOX_TRY(run_sigma(h, p, dev[0], dev[1], dev[2], dev[3], dev[4], stream));   // SOX(v, W0)
    SOX_TRY(run_sigma(h, p, dev[0], dev[1], Wd, dev[2], part, stream));         // SOX(W_d, v)
    sox::launch_add_f64(dev[4], part, dev[4], nsig, s);
    ++h->launches;
    SOX_CUDA_TRY(cudaGetLastError());
    if (host[4]) {
      SOX_CUDA_TRY(cudaMemcpyAsync(Sigma, dev[4], 8 * (size_t)nsig, cudaMemcpyDeviceToHost, s));
      SOX_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return Status::ok();
  }();
  return finish(h, st);
}

int sox_pi0(sox_handle h, const sox_problem *p, const double *G, const double *X,
            const double *w, double *Pi0, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(validate(p));
    if (!G || !X || !w || !Pi0) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const Dims d = dims_of(p);
    Call call(h, stream);
    Staged sG, sX, sw, oP;
    SOX_TRY(call.input(G, (size_t)d.S * d.T * d.nn(), &sG));
    SOX_TRY(call.input(X, (size_t)d.N * d.n, &sX));
    SOX_TRY(call.input(w, (size_t)d.T, &sw));
    SOX_TRY(call.output(Pi0, (size_t)d.S * d.N * d.N, &oP));
    const size_t gpq = (size_t)d.T * d.N * d.N, gr = (size_t)d.T * d.N * d.n;
    Arena ar;
    SOX_TRY(call.begin(sox::aligned_bytes(gpq, 8) + sox::aligned_bytes(gr, 8), &ar));
    double *GPQ = ar.take<double>(gpq);
    double *GR = ar.take<double>(gr);
    cudaStream_t s = call.stream();
    for (int sp = 0; sp < d.S; ++sp) {
      const double *Gs = sG.in + (long long)sp * d.T * d.nn();
      GemmF64 g;
      g.M = d.N; g.Nc = d.n; g.K = d.n; g.batch = d.T;
      g.A = sX.in; g.ai = d.n; g.ak = 1;
      g.B = Gs; g.sB = d.nn(); g.bk = d.n; g.bj = 1;
      g.C = GR; g.sC = (long long)d.N * d.n; g.ci = d.n; g.cj = 1;
      sox::ProfScope ps0(h, "project_f64", s, 2);
      sox::launch_gemm_f64(g, s);
      GemmF64 q;
      q.M = d.N; q.Nc = d.N; q.K = d.n; q.batch = d.T;
      q.A = GR; q.sA = (long long)d.N * d.n; q.ai = d.n; q.ak = 1;
      q.B = sX.in; q.bk = 1; q.bj = d.n;
      q.C = GPQ; q.sC = (long long)d.N * d.N; q.ci = d.N; q.cj = 1;
      sox::launch_gemm_f64(q, s);
      sox::ProfScope ps1(h, "pi0_reduce", s);
      sox::launch_pi0_reduce(GPQ, sw.in, d.N, d.T, oP.out + (long long)sp * d.N * d.N, s);
    }
    return call.end();
  }();
  return finish(h, st);
}

int sox_w_static(sox_handle h, const sox_problem *p, const double *V, const double *Pi,
                 double *W0, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(validate(p));
    if (!V || !Pi || !W0) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const int N = p->N;
    Call call(h, stream);
    Staged sV, sP, oW;
    SOX_TRY(call.input(V, (size_t)N * N, &sV));
    SOX_TRY(call.input(Pi, (size_t)N * N, &sP));
    SOX_TRY(call.output(W0, (size_t)N * N, &oW));
    Arena ar;
    SOX_TRY(call.begin(sox::aligned_bytes((size_t)2 * N * N, 8) + 256, &ar));
    double *Aug = ar.take<double>((size_t)2 * N * N);
    int *info = ar.take<int>(4);
    cudaStream_t s = call.stream();
    SOX_CUDA_TRY(cudaMemsetAsync(info, 0, 4 * sizeof(int), s));
    {
      sox::ProfScope ps(h, "w_static_gj", s, 3 + 2 * N);
      sox::launch_build_gj_system(sV.in, sP.in, Aug, N, s);
      for (int k = 0; k < N; ++k) sox::launch_gj_step(Aug, N, k, info, s);
      sox::launch_copy_right_half(Aug, oW.out, N, s);
    }
    int hinfo[4] = {0, 0, 0, 0};
    SOX_CUDA_TRY(cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, s));
    SOX_CUDA_TRY(cudaStreamSynchronize(s));
    if (hinfo[1]) return {SOX_ERR_INVALID_ARG, "1 - V Pi is singular"};
    return call.end();
  }();
  return finish(h, st);
}

int phi_sox(sox_handle h, const sox_problem *p, const double *G, const double *X,
            const double *V, const double *w, double *phi, double *Sigma_out, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(validate(p));
    if (!G || !X || !V || !w || !phi) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const Dims d = dims_of(p);
    const size_t nsig = (size_t)d.S * d.T * d.nn();
    Call call(h, stream);
    Staged sG, sX, sV, sw, oPhi, oS;
    SOX_TRY(call.input(G, nsig, &sG));
    SOX_TRY(call.input(X, (size_t)d.N * d.n, &sX));
    SOX_TRY(call.input(V, (size_t)d.N * d.N, &sV));
    SOX_TRY(call.input(w, (size_t)d.T, &sw));
    SOX_TRY(call.output(phi, (size_t)d.S, &oPhi));
    SOX_TRY(call.output(Sigma_out, nsig, &oS));
    Arena ar;
    SOX_TRY(call.begin(sigma_bytes(h, d, false) + sox::aligned_bytes(nsig, 8) +
                           sox::aligned_bytes((size_t)d.S * d.T, 8), &ar));
    double *sig = oS.out ? oS.out : ar.take<double>(nsig);
    double *part = ar.take<double>((size_t)d.S * d.T);
    cudaStream_t s = call.stream();
    SOX_TRY(sigma_any(h, d, sG.in, sX.in, sV.in, sV.in, sig, ar, s));
    {
      sox::ProfScope ps(h, "phi_trace", s, 2);
      sox::launch_trace_sigma_gminus(sig, sG.in, d.n, d.T, d.S, part, s);
      sox::launch_phi_finish(part, sw.in, d.T, d.S, oPhi.out, s);
    }
    return call.end();
  }();
  return finish(h, st);
}

int phi_sox_backward(sox_handle h, const sox_problem *p, const double *G, const double *X,
                     const double *V, const double *w, const double *dphi, double *dG,
                     double *dX, double *dV, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(validate(p));
    if (!G || !X || !V || !w || !dphi) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const Dims d = dims_of(p);
    const size_t nsig = (size_t)d.S * d.T * d.nn();
    Call call(h, stream);
    Staged sG, sX, sV, sw, sd, oG, oX, oV;
    SOX_TRY(call.input(G, nsig, &sG));
    SOX_TRY(call.input(X, (size_t)d.N * d.n, &sX));
    SOX_TRY(call.input(V, (size_t)d.N * d.N, &sV));
    SOX_TRY(call.input(w, (size_t)d.T, &sw));
    SOX_TRY(call.input(dphi, (size_t)d.S, &sd));
    SOX_TRY(call.output(dG, nsig, &oG));
    SOX_TRY(call.output(dX, (size_t)d.N * d.n, &oX));
    SOX_TRY(call.output(dV, (size_t)d.N * d.N, &oV));
    if (dG && !sox::v_range_is_full(h, d.n))
      return {SOX_ERR_UNSUPPORTED, "dG needs the whole Sigma (the identity dPhi/dG = -w Sigma(beta - tau)^T does not "
                                   "hold for a partial v range); clear the v range or request dX / dV only"};
    size_t need = 0;
    if (dG) need = sigma_bytes(h, d, false) + sox::aligned_bytes(nsig, 8);
    const bool tc_adj = (h->precision == SOX_PREC_F16X2);
    if (dX || dV)
      need = std::max(need, tc_adj ? sox::adjoint_tc_bytes(h, d.n, d.N, d.T, d.S)
                                   : sox::adjoint_bytes(h, d.n, d.N, d.T, d.S, nullptr));
    Arena ar;
    SOX_TRY(call.begin(need, &ar));
    cudaStream_t s = call.stream();
    if (oG.out) {
      // dPhi/dG_rt(tau_j) = -w_j Sigma_tr(beta - tau_j) (bare SOX on a mirror-symmetric grid)
      Arena a2 = ar;
      double *sig = a2.take<double>(nsig);
      SOX_TRY(sigma_any(h, d, sG.in, sX.in, sV.in, sV.in, sig, a2, s));
      sox::ProfScope ps(h, "dG_identity", s);
      sox::launch_dG_from_sigma(sig, sw.in, sd.in, d.n, d.T, d.S, oG.out, s);
    }
    if (oX.out || oV.out) {
      Arena a3 = ar;
      if (tc_adj)
        SOX_TRY(sox::phi_adjoint_xv_tc(h, d.n, d.N, d.T, d.S, sG.in, sX.in, sV.in, sw.in, sd.in, oX.out, oV.out, a3,
                                       s));
      else
        SOX_TRY(sox::phi_adjoint_xv_f64(h, d.n, d.N, d.T, d.S, sG.in, sX.in, sV.in, sw.in, sd.in, oX.out, oV.out,
                                      a3, s));
    }
    return call.end();
  }();
  return finish(h, st);
}

int phi_sox_grad_G(sox_handle h, const sox_problem *p, const double *Sigma, const double *w, const double *dphi,
                   double *dG, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(validate(p));
    if (!Sigma || !w || !dphi || !dG) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    if (Sigma == dG) return {SOX_ERR_INVALID_ARG, "dG must not alias Sigma"};
    SOX_TRY(bind_device(h));
    const Dims d = dims_of(p);
    const size_t nsig = (size_t)d.S * d.T * d.nn();
    Call call(h, stream);
    Staged sS, sw, sd, oG;
    SOX_TRY(call.input(Sigma, nsig, &sS));
    SOX_TRY(call.input(w, (size_t)d.T, &sw));
    SOX_TRY(call.input(dphi, (size_t)d.S, &sd));
    SOX_TRY(call.output(dG, nsig, &oG));
    Arena ar;
    SOX_TRY(call.begin(0, &ar));
    sox::ProfScope ps(h, "dG_identity", call.stream());
    sox::launch_dG_from_sigma(sS.in, sw.in, sd.in, d.n, d.T, d.S, oG.out, call.stream());
    return call.end();
  }();
  return finish(h, st);
}

int sox_w_dynamic(sox_handle h, const sox_problem *p, const double *G, const double *X, const double *V,
                  const double *T_fwd, int n_omega, double *Wd, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    if (!G || !X || !V || !T_fwd || !Wd) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    if (n_omega < 1 || n_omega > SOX_MAX_N_TAU) return {SOX_ERR_SHAPE, "n_omega out of range [1, SOX_MAX_N_TAU]"};
    const bool solid = p && (p->dtype == SOX_COMPLEX128 || p->nk[0] * p->nk[1] * p->nk[2] != 1);
    if (solid) {
      SOX_TRY(validate(p, false));
      if (p->dtype != SOX_COMPLEX128)
        return {SOX_ERR_UNSUPPORTED, "k-point meshes need complex data (SOX_COMPLEX128)"};
    } else {
      SOX_TRY(validate(p));
    }
    const int nk = p->nk[0] * p->nk[1] * p->nk[2];
    if (p->nk[0] > 8 || p->nk[1] > 8 || p->nk[2] > 8) return {SOX_ERR_SHAPE, "mesh sides above 8"};
    if ((long long)nk * n_omega > 65535) return {SOX_ERR_SHAPE, "more than 65535 (q, Omega) systems"};
    SOX_TRY(bind_device(h));
    const size_t c = solid ? 2 : 1;
    const size_t nn = (size_t)p->n * p->n, NN = (size_t)p->N * p->N;
    Call call(h, stream);
    Staged sG, sX, sV, sF, oW;
    SOX_TRY(call.input(G, c * p->n_spin * nk * p->n_tau * nn, &sG));
    SOX_TRY(call.input(X, c * nk * p->N * p->n, &sX));
    SOX_TRY(call.input(V, c * nk * NN, &sV));
    SOX_TRY(call.input(T_fwd, 2 * (size_t)n_omega * p->n_tau, &sF));
    SOX_TRY(call.output(Wd, c * nk * n_omega * NN, &oW));
    Arena ar;
    SOX_TRY(call.begin(sox::w_dynamic_bytes(p, n_omega), &ar));
    SOX_TRY(sox::w_dynamic(h, p, n_omega, sG.in, sX.in, sV.in, sF.in, oW.out, ar, call.stream()));
    return call.end();
  }();
  return finish(h, st);
}

int sosex_dynamic_sigma(sox_handle h, const sox_problem *p, const double *G, const double *X,
                        const double *V, const double *Wd, const double *T_fwd,
                        const double *T_inv, int n_omega, double *Sigma, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    if (!G || !X || !V || !Wd || !T_fwd || !T_inv || !Sigma) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    if (n_omega < 1 || n_omega > SOX_MAX_N_TAU) return {SOX_ERR_SHAPE, "n_omega out of range [1, SOX_MAX_N_TAU]"};
    if (p && (p->dtype == SOX_COMPLEX128 || p->nk[0] * p->nk[1] * p->nk[2] != 1)) {
      // solids (complex data, any k-mesh): momentum-resolved chain in FP64 complex
      SOX_TRY(validate(p, false));
      if (p->dtype != SOX_COMPLEX128)
        return {SOX_ERR_UNSUPPORTED, "k-point meshes need complex data (SOX_COMPLEX128)"};
      SOX_TRY(bind_device(h));
      const int nk = p->nk[0] * p->nk[1] * p->nk[2];
      const size_t nn = (size_t)p->n * p->n, NN = (size_t)p->N * p->N;
      Call call(h, stream);
      Staged sG, sX, sV, sW, sF, sI, oS;
      SOX_TRY(call.input(G, 2 * (size_t)p->n_spin * nk * p->n_tau * nn, &sG));
      SOX_TRY(call.input(X, 2 * (size_t)nk * p->N * p->n, &sX));
      SOX_TRY(call.input(V, 2 * (size_t)nk * NN, &sV));
      SOX_TRY(call.input(Wd, 2 * (size_t)nk * n_omega * NN, &sW));
      SOX_TRY(call.input(T_fwd, 2 * (size_t)n_omega * p->n_tau, &sF));
      SOX_TRY(call.input(T_inv, 2 * (size_t)n_omega * p->n_tau, &sI));
      SOX_TRY(call.output(Sigma, 2 * (size_t)p->n_spin * nk * p->n_tau * nn, &oS));
      Arena ar;
      if (h->precision == SOX_PREC_F16X2) {
        SOX_TRY(call.begin(std::max(sox::kpoint_tc_bytes(h, p, false), sox::kpoint_dynamic_tc_bytes(h, p, n_omega)),
                           &ar));
        {
          Arena a1 = ar;
          SOX_TRY(sox::kpoint_sigma_tc(h, p, sG.in, sX.in, sV.in, sV.in, oS.out, a1, call.stream()));
        }
        Arena a2 = ar;
        SOX_TRY(sox::kpoint_dynamic_tc(h, p, n_omega, sG.in, sX.in, sV.in, sW.in, sF.in, sI.in, oS.out, a2,
                                       call.stream()));
        return call.end();
      }
      const sox::KpointPlan pl = sox::kpoint_plan(h, p->n, p->N, p->n_tau, p->n_spin, p->nk);
      SOX_TRY(call.begin(std::max(pl.bytes, sox::kpoint_dynamic_bytes(h, p->n, p->N, p->n_tau, n_omega, p->nk, nullptr)),
                         &ar));
      {
        Arena a1 = ar;
        SOX_TRY(sox::kpoint_sigma_f64(h, p, sG.in, sX.in, sV.in, sV.in, oS.out, a1, call.stream()));
      }
      Arena a2 = ar;
      SOX_TRY(sox::kpoint_dynamic_add_f64(h, p, n_omega, sG.in, sX.in, sV.in, sW.in, sF.in, sI.in, oS.out, a2,
                                          call.stream()));
      return call.end();
    }
    SOX_TRY(validate(p));
    SOX_TRY(bind_device(h));
    const Dims d = dims_of(p);
    const size_t nsig = (size_t)d.S * d.T * d.nn();
    Call call(h, stream);
    Staged sG, sX, sV, sW, sF, sI, oS;
    SOX_TRY(call.input(G, nsig, &sG));
    SOX_TRY(call.input(X, (size_t)d.N * d.n, &sX));
    SOX_TRY(call.input(V, (size_t)d.N * d.N, &sV));
    SOX_TRY(call.input(Wd, (size_t)n_omega * d.N * d.N, &sW));
    SOX_TRY(call.input(T_fwd, 2 * (size_t)n_omega * d.T, &sF));
    SOX_TRY(call.input(T_inv, 2 * (size_t)n_omega * d.T, &sI));
    SOX_TRY(call.output(Sigma, nsig, &oS));
    Arena ar;
    const bool tc_dyn = (h->precision == SOX_PREC_F16X2);
    const size_t dyn_bytes = tc_dyn ? sox::dynamic_tc_bytes(h, d.n, d.N, d.T, d.S, n_omega)
                                    : sox::dynamic_bytes(d.n, d.N, d.T, n_omega);
    SOX_TRY(call.begin(std::max(sigma_bytes(h, d, false), dyn_bytes), &ar));
    cudaStream_t s = call.stream();
    {  // SOX(v, v): the static part, in the handle's precision
      Arena a1 = ar;
      SOX_TRY(sigma_any(h, d, sG.in, sX.in, sV.in, sV.in, oS.out, a1, s));
    }
    Arena a2 = ar;
    if (tc_dyn)
      SOX_TRY(sox::dynamic_sigma_add_tc(h, d.n, d.N, d.T, d.S, n_omega, sG.in, sX.in, sV.in, sW.in, sF.in, sI.in,
                                        oS.out, a2, s));
    else
      SOX_TRY(sox::dynamic_sigma_add_f64(h, d.n, d.N, d.T, d.S, n_omega, sG.in, sX.in, sV.in, sW.in, sF.in, sI.in,
                                         oS.out, a2, s));
    return call.end();
  }();
  return finish(h, st);
}

// The uneven batch of molecules, with Phi per instance when w and phi are given.  Split
// precision: every instance's chain up to A and after D runs per instance, and the fused
// B / C / Hadamard step of one tau chunk of every instance is one persistent launch
// (tc_sigma_batch).  FP64 (or a single instance): the instances run in turn.
Status batch_call(sox_handle h, int count, const sox_problem *probs, const double *const *G,
                  const double *const *X, const double *const *V, const double *const *w, double *const *phi,
                  double *const *Sigma, void *stream) {
  if (count < 1 || !probs || !G || !X || !V || !Sigma) return {SOX_ERR_INVALID_ARG, "bad batch arrays"};
  const bool with_phi = (w != nullptr || phi != nullptr);
  if (with_phi && (!w || !phi)) return {SOX_ERR_INVALID_ARG, "w and phi go together"};
  bool solid = false;
  for (int i = 0; i < count; ++i)
    solid = solid || probs[i].dtype == SOX_COMPLEX128 || probs[i].nk[0] * probs[i].nk[1] * probs[i].nk[2] != 1;
  if (solid && !with_phi) {   // solids: each instance through its own chain
    for (int i = 0; i < count; ++i) {
      Status st = run_sigma(h, &probs[i], G[i], X[i], V[i], V[i], Sigma[i], stream);
      if (!st.good()) {
        st.msg = "instance " + std::to_string(i) + ": " + st.msg;
        return st;
      }
    }
    return Status::ok();
  }
  std::vector<Dims> d(count);
  for (int i = 0; i < count; ++i) {
    Status v = validate(&probs[i]);   // molecules (real data, one k point)
    if (v.good() && (!G[i] || !X[i] || !V[i] || !Sigma[i] || (with_phi && (!w[i] || !phi[i]))))
      v = {SOX_ERR_INVALID_ARG, "a required tensor pointer is NULL"};
    if (!v.good()) {
      v.msg = "instance " + std::to_string(i) + ": " + v.msg;
      return v;
    }
    d[i] = dims_of(&probs[i]);
  }
  SOX_TRY(bind_device(h));
  const bool fused = (h->precision == SOX_PREC_F16X2 && count > 1);
  std::vector<int> n(count), N(count), T(count), S(count);
  std::vector<Staged> sG(count), sX(count), sV(count), sw(count), sS(count), sP(count);
  Call call(h, stream);
  size_t part_bytes = 0, compute = 0;
  for (int i = 0; i < count; ++i) {
    n[i] = d[i].n; N[i] = d[i].N; T[i] = d[i].T; S[i] = d[i].S;
    const size_t nsig = (size_t)d[i].S * d[i].T * d[i].nn();
    SOX_TRY(call.input(G[i], nsig, &sG[i]));
    SOX_TRY(call.input(X[i], (size_t)d[i].N * d[i].n, &sX[i]));
    SOX_TRY(call.input(V[i], (size_t)d[i].N * d[i].N, &sV[i]));
    SOX_TRY(call.output(Sigma[i], nsig, &sS[i]));
    if (with_phi) {
      SOX_TRY(call.input(w[i], (size_t)d[i].T, &sw[i]));
      SOX_TRY(call.output(phi[i], (size_t)d[i].S, &sP[i]));
      part_bytes += sox::aligned_bytes((size_t)d[i].S * d[i].T, 8);
    }
    if (!fused) compute = std::max(compute, sigma_bytes(h, d[i], false));
  }
  if (fused) compute = sox::tc_sigma_batch_bytes(h, count, n.data(), N.data(), T.data(), S.data());
  Arena ar;
  SOX_TRY(call.begin(compute + part_bytes, &ar));
  cudaStream_t s = call.stream();
  std::vector<double *> part(count, nullptr);
  if (with_phi)
    for (int i = 0; i < count; ++i) part[i] = ar.take<double>((size_t)d[i].S * d[i].T);
  if (fused) {
    std::vector<const double *> Gd(count), Xd(count), Vd(count);
    std::vector<double *> Sd(count);
    for (int i = 0; i < count; ++i) {
      Gd[i] = sG[i].in; Xd[i] = sX[i].in; Vd[i] = sV[i].in; Sd[i] = sS[i].out;
    }
    Arena a = ar;
    SOX_TRY(sox::tc_sigma_batch(h, count, n.data(), N.data(), T.data(), S.data(), Gd.data(), Xd.data(), Vd.data(),
                                Sd.data(), a, s));
  } else {
    for (int i = 0; i < count; ++i) {
      Arena a = ar;
      Status st = sigma_any(h, d[i], sG[i].in, sX[i].in, sV[i].in, sV[i].in, sS[i].out, a, s);
      if (!st.good()) {
        st.msg = "instance " + std::to_string(i) + ": " + st.msg;
        return st;
      }
    }
  }
  if (with_phi) {
    sox::ProfScope ps(h, "phi_trace", s, 2 * count);
    for (int i = 0; i < count; ++i) {
      sox::launch_trace_sigma_gminus(sS[i].out, sG[i].in, d[i].n, d[i].T, d[i].S, part[i], s);
      sox::launch_phi_finish(part[i], sw[i].in, d[i].T, d[i].S, sP[i].out, s);
    }
  }
  return call.end();
}

int sox_sigma_batch(sox_handle h, int count, const sox_problem *probs, const double *const *G,
                    const double *const *X, const double *const *V, double *const *Sigma,
                    void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  if (count < 0) return finish(h, {SOX_ERR_INVALID_ARG, "bad batch arrays"});
  if (count == 0) return finish(h, Status::ok());
  return finish(h, batch_call(h, count, probs, G, X, V, nullptr, nullptr, Sigma, stream));
}

int phi_sox_batch(sox_handle h, int count, const sox_problem *probs, const double *const *G, const double *const *X,
                  const double *const *V, const double *const *w, double *const *phi, double *const *Sigma,
                  void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  if (count < 0 || (count > 0 && (!w || !phi))) return finish(h, {SOX_ERR_INVALID_ARG, "bad batch arrays"});
  if (count == 0) return finish(h, Status::ok());
  return finish(h, batch_call(h, count, probs, G, X, V, w, phi, Sigma, stream));
}

// ---------------------------------------------------------------------------
// Batch plans: the sox_sigma sequence of an uneven batch recorded once into a
// CUDA graph (own handle and workspace), replayed with one launch.
// ---------------------------------------------------------------------------
struct sox_plan_s {
  sox_handle ih = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int count = 0;
};

static void plan_free(sox_plan p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->ih) sox_destroy(p->ih);
  delete p;
}

static Status plan_device_tensor(sox_handle h, const void *ptr, const char *what) {
  if (!ptr) return {SOX_ERR_INVALID_ARG, std::string(what) + " is NULL"};
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return {SOX_ERR_INVALID_ARG, std::string(what) + ": not a device pointer"};
  }
  if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != h->device)
    return {SOX_ERR_INVALID_ARG, std::string(what) + ": batch plans take device memory of the handle's GPU"};
  return Status::ok();
}

int sox_sigma_batch_plan(sox_handle h, int count, const sox_problem *probs, const double *const *G,
                         const double *const *X, const double *const *V, double *const *Sigma, sox_plan *out) {
  if (!h || !out) return SOX_ERR_INVALID_ARG;
  *out = nullptr;
  sox_plan plan = nullptr;
  cudaStream_t cs = nullptr;
  Status st = [&]() -> Status {
    if (count < 1 || !probs || !G || !X || !V || !Sigma) return {SOX_ERR_INVALID_ARG, "bad batch arrays"};
    SOX_TRY(bind_device(h));
    for (int i = 0; i < count; ++i) {
      Status v = validate(&probs[i]);   // molecules (real data, one k point)
      if (!v.good()) {
        v.msg = "instance " + std::to_string(i) + ": " + v.msg;
        return v;
      }
      SOX_TRY(plan_device_tensor(h, G[i], "G"));
      SOX_TRY(plan_device_tensor(h, X[i], "X"));
      SOX_TRY(plan_device_tensor(h, V[i], "V"));
      SOX_TRY(plan_device_tensor(h, Sigma[i], "Sigma"));
    }
    plan = new (std::nothrow) sox_plan_s();
    if (!plan) return {SOX_ERR_OOM, "plan allocation failed"};
    plan->count = count;
    sox_options o{h->precision, h->device, h->spin_limit, (long long)h->ws_limit, h->autotune ? 0 : 1};
    const int rc = sox_create(&plan->ih, &o);
    if (rc != SOX_OK) return {rc, "could not create the plan's handle"};
    plan->ih->v0 = h->v0;   // the plan keeps the v range of its handle at creation
    plan->ih->v1 = h->v1;
    SOX_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    // eager pass: sizes the plan's workspace for the largest instance and settles the
    // autotuned kernel choices, so that the recorded pass allocates and times nothing
    SOX_TRY(batch_call(plan->ih, count, probs, G, X, V, nullptr, nullptr, Sigma, cs));
    SOX_CUDA_TRY(cudaStreamSynchronize(cs));
    SOX_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    Status rec = batch_call(plan->ih, count, probs, G, X, V, nullptr, nullptr, Sigma, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &g);
    if (!rec.good()) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return rec;
    }
    if (ec != cudaSuccess) return {SOX_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ec)};
    plan->graph = g;
    SOX_CUDA_TRY(cudaGraphInstantiate(&plan->exec, plan->graph, 0));
    return Status::ok();
  }();
  if (cs) cudaStreamDestroy(cs);
  if (!st.good()) {
    plan_free(plan);
    return finish(h, st);
  }
  *out = plan;
  return finish(h, st);
}

int sox_plan_launch(sox_plan plan, void *stream) {
  if (!plan || !plan->exec) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(bind_device(plan->ih));
    SOX_CUDA_TRY(cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)));
    return Status::ok();
  }();
  return finish(plan->ih, st);
}

int sox_plan_check_device(sox_plan plan) {
  if (!plan) return SOX_ERR_INVALID_ARG;
  return sox_check_device(plan->ih);
}

const char *sox_plan_last_error(sox_plan plan) { return plan ? sox_last_error(plan->ih) : "plan is NULL"; }

int sox_plan_destroy(sox_plan plan) {
  if (!plan) return SOX_ERR_INVALID_ARG;
  if (plan->ih) {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(plan->ih->device);
    cudaDeviceSynchronize();
    if (prev >= 0) cudaSetDevice(prev);
  }
  plan_free(plan);
  return SOX_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// The self-consistent loop around Sigma for molecules (Sec. II A)
// ----------------------------------------------------------------------------
namespace {
Status loop_problem(const sox_problem *p) {
  SOX_TRY(validate(p));
  if (p->dtype != SOX_REAL64) return {SOX_ERR_UNSUPPORTED, "the loop steps take real molecular data"};
  return Status::ok();
}
}  // namespace

int sox_dyson(sox_handle h, const sox_problem *p, int n_w, const double *omegas, double mu, const double *F,
              const double *Sigma_iw, double *G_iw, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(loop_problem(p));
    if (n_w < 1 || n_w > (1 << 20)) return {SOX_ERR_SHAPE, "n_w out of range [1, 2^20]"};
    if (!omegas || !F || !G_iw) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const size_t nn = (size_t)p->n * p->n, S = p->n_spin;
    Call call(h, stream);
    Staged sw, sF, sS, oG;
    SOX_TRY(call.input(omegas, (size_t)n_w, &sw));
    SOX_TRY(call.input(F, S * nn, &sF));
    SOX_TRY(call.input(Sigma_iw, 2 * S * n_w * nn, &sS));
    SOX_TRY(call.output(G_iw, 2 * S * n_w * nn, &oG));
    Arena ar;
    SOX_TRY(call.begin(sox::dyson_bytes(p->n, n_w, p->n_spin), &ar));
    SOX_TRY(sox::dyson(h, p->n, n_w, p->n_spin, sw.in, mu, sF.in, sS.in, oG.out, ar, call.stream()));
    return call.end();
  }();
  return finish(h, st);
}

int sox_green_tails(sox_handle h, const sox_problem *p, double mu, const double *F, const double *Sigma_tau,
                    double *tails, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(loop_problem(p));
    if (!F || !tails) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const size_t nn = (size_t)p->n * p->n, S = p->n_spin;
    Call call(h, stream);
    Staged sF, sS, oT;
    SOX_TRY(call.input(F, S * nn, &sF));
    SOX_TRY(call.input(Sigma_tau, S * p->n_tau * nn, &sS));
    SOX_TRY(call.output(tails, 3 * S * nn, &oT));
    Arena ar;
    SOX_TRY(call.begin(0, &ar));
    sox::ProfScope ps(h, "green_tails", call.stream());
    sox::launch_green_tails(sF.in, mu, sS.in, p->n, p->n_tau, p->n_spin, oT.out, call.stream());
    SOX_CUDA_TRY(cudaGetLastError());
    return call.end();
  }();
  return finish(h, st);
}

int sox_iw_to_tau(sox_handle h, const sox_problem *p, int n_w, const double *omegas, const double *G_iw,
                  const double *tails, int n_t, const double *tau, double *G_tau, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(loop_problem(p));
    if (n_w < 1 || n_t < 1 || n_t > SOX_MAX_N_TAU) return {SOX_ERR_SHAPE, "n_w or n_t out of range"};
    if (!omegas || !G_iw || !tails || !tau || !G_tau) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const size_t nn = (size_t)p->n * p->n, S = p->n_spin;
    Call call(h, stream);
    Staged sw, sG, sT, st_, oG;
    SOX_TRY(call.input(omegas, (size_t)n_w, &sw));
    SOX_TRY(call.input(G_iw, 2 * S * n_w * nn, &sG));
    SOX_TRY(call.input(tails, 3 * S * nn, &sT));
    SOX_TRY(call.input(tau, (size_t)n_t, &st_));
    SOX_TRY(call.output(G_tau, S * n_t * nn, &oG));
    Arena ar;
    SOX_TRY(call.begin(0, &ar));
    sox::ProfScope ps(h, "iw_to_tau", call.stream());
    sox::launch_iw_to_tau(sG.in, sw.in, n_w, sT.in, st_.in, n_t, p->n, p->n_spin, p->beta, oG.out, call.stream());
    SOX_CUDA_TRY(cudaGetLastError());
    return call.end();
  }();
  return finish(h, st);
}

int sox_tau_to_iw(sox_handle h, const sox_problem *p, int n_w, const double *T_w, const double *F_tau, double *F_iw,
                  void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(loop_problem(p));
    if (n_w < 1 || n_w > (1 << 20)) return {SOX_ERR_SHAPE, "n_w out of range [1, 2^20]"};
    if (!T_w || !F_tau || !F_iw) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const size_t nn = (size_t)p->n * p->n, S = p->n_spin;
    Call call(h, stream);
    Staged sT, sF, oF;
    SOX_TRY(call.input(T_w, 2 * (size_t)n_w * p->n_tau, &sT));
    SOX_TRY(call.input(F_tau, S * p->n_tau * nn, &sF));
    SOX_TRY(call.output(F_iw, 2 * S * n_w * nn, &oF));
    Arena ar;
    SOX_TRY(call.begin(0, &ar));
    sox::ProfScope ps(h, "tau_to_iw", call.stream());
    sox::launch_tau_to_iw(sT.in, sF.in, n_w, p->n_tau, p->n, p->n_spin, oF.out, call.stream());
    SOX_CUDA_TRY(cudaGetLastError());
    return call.end();
  }();
  return finish(h, st);
}

int sox_find_mu(sox_handle h, const sox_problem *p, int n_w, const double *omegas, double target, const double *F,
                const double *Sigma_iw, const double *Sigma_tau, double lo, double hi, double tol, int max_iter,
                double *mu) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(loop_problem(p));
    if (n_w < 1 || n_w > (1 << 20)) return {SOX_ERR_SHAPE, "n_w out of range [1, 2^20]"};
    if (!omegas || !F || !mu) return {SOX_ERR_INVALID_ARG, "NULL pointer"};
    if (!(hi > lo) || !(tol > 0.0) || max_iter < 1) return {SOX_ERR_INVALID_ARG, "need lo < hi, tol > 0, max_iter >= 1"};
    SOX_TRY(bind_device(h));
    const size_t nn = (size_t)p->n * p->n, S = p->n_spin;
    Call call(h, nullptr);
    Staged sw, sF, sSi, sSt;
    SOX_TRY(call.input(omegas, (size_t)n_w, &sw));
    SOX_TRY(call.input(F, S * nn, &sF));
    SOX_TRY(call.input(Sigma_iw, 2 * S * n_w * nn, &sSi));
    SOX_TRY(call.input(Sigma_tau, S * p->n_tau * nn, &sSt));
    Arena ar;
    const size_t extra = sox::aligned_bytes(2 * S * n_w * nn, 8) + sox::aligned_bytes(3 * S * nn, 8) + 4096;
    SOX_TRY(call.begin(sox::dyson_bytes(p->n, n_w, p->n_spin) + extra, &ar));
    cudaStream_t s = call.stream();
    double *Giw = ar.take<double>(2 * S * n_w * nn), *tails = ar.take<double>(3 * S * nn);
    double *count = ar.take<double>(1);
    if (!count) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
    // bisection on the electron count sum_s Tr gamma^s(mu), which rises with mu (Sec. II A)
    for (int it = 0; it < max_iter && hi - lo >= tol; ++it) {
      const double mid = 0.5 * (lo + hi);
      Arena a2 = ar;
      SOX_TRY(sox::dyson(h, p->n, n_w, p->n_spin, sw.in, mid, sF.in, sSi.in, Giw, a2, s));
      sox::launch_green_tails(sF.in, mid, sSt.in, p->n, p->n_tau, p->n_spin, tails, s);
      SOX_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(double), s));
      sox::launch_trace_gamma(Giw, sw.in, n_w, tails, p->n, p->n_spin, p->beta, count, s);
      h->launches += 3;
      double c = 0.0;
      SOX_CUDA_TRY(cudaMemcpyAsync(&c, count, sizeof(double), cudaMemcpyDeviceToHost, s));
      SOX_CUDA_TRY(cudaStreamSynchronize(s));
      if (c < target)
        lo = mid;
      else
        hi = mid;
    }
    *mu = 0.5 * (lo + hi);
    return call.end();
  }();
  return finish(h, st);
}

int sox_sigma_hf(sox_handle h, const sox_problem *p, const double *X, const double *V, const double *gamma,
                 const double *H0, double *Sigma_hf, double *F, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(loop_problem(p));
    if (!X || !V || !gamma || !Sigma_hf) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const size_t nn = (size_t)p->n * p->n, S = p->n_spin, N = p->N;
    Call call(h, stream);
    if (F && !H0) return {SOX_ERR_INVALID_ARG, "F needs H0"};
    Staged sX, sV, sg, sH, oS, oF;
    SOX_TRY(call.input(X, N * p->n, &sX));
    SOX_TRY(call.input(V, N * N, &sV));
    SOX_TRY(call.input(gamma, S * nn, &sg));
    SOX_TRY(call.input(H0, nn, &sH));
    SOX_TRY(call.output(Sigma_hf, S * nn, &oS));
    SOX_TRY(call.output(F, S * nn, &oF));
    Arena ar;
    SOX_TRY(call.begin(sox::aligned_bytes(N + S * N * p->n, 8) + sox::aligned_bytes(S * N * N, 8), &ar));
    double *d = ar.take<double>(N + S * N * p->n), *Gam = ar.take<double>(S * N * N);
    if (!Gam) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
    sox::ProfScope ps(h, "sigma_hf", call.stream(), 2 + 2 * p->n_spin);
    sox::launch_sigma_hf(sX.in, sV.in, sg.in, p->N, p->n, p->n_spin, d, Gam, oS.out, call.stream());
    for (int sp = 0; oF.out && sp < p->n_spin; ++sp)   // F[s] = H0 + Sigma_HF[s]
      sox::launch_add_f64(sH.in, oS.out + sp * nn, oF.out + sp * nn, (long long)nn, call.stream());
    SOX_CUDA_TRY(cudaGetLastError());
    return call.end();
  }();
  return finish(h, st);
}

int sox_density_matrix(sox_handle h, const sox_problem *p, const double *G_tau, double *gamma, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(loop_problem(p));
    if (!G_tau || !gamma) return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const size_t nn = (size_t)p->n * p->n, S = p->n_spin;
    Call call(h, stream);
    Staged sG, og;
    SOX_TRY(call.input(G_tau, S * p->n_tau * nn, &sG));
    SOX_TRY(call.output(gamma, S * nn, &og));
    Arena ar;
    SOX_TRY(call.begin(0, &ar));
    sox::ProfScope ps(h, "density_matrix", call.stream());
    sox::launch_gamma_from_tau(sG.in, p->n, p->n_tau, p->n_spin, og.out, call.stream());
    SOX_CUDA_TRY(cudaGetLastError());
    return call.end();
  }();
  return finish(h, st);
}

int sox_gm_energies(sox_handle h, const sox_problem *p, const double *H0, const double *Sigma_hf, const double *gamma,
                    const double *Sigma_tau, const double *G_tau, const double *w, double *E, void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    SOX_TRY(loop_problem(p));
    if (!H0 || !Sigma_hf || !gamma || !Sigma_tau || !G_tau || !w || !E)
      return {SOX_ERR_INVALID_ARG, "NULL tensor pointer"};
    SOX_TRY(bind_device(h));
    const size_t nn = (size_t)p->n * p->n, S = p->n_spin, T = p->n_tau;
    Call call(h, stream);
    Staged sH, sS, sg, sSt, sG, sw, oE;
    SOX_TRY(call.input(H0, nn, &sH));
    SOX_TRY(call.input(Sigma_hf, S * nn, &sS));
    SOX_TRY(call.input(gamma, S * nn, &sg));
    SOX_TRY(call.input(Sigma_tau, S * T * nn, &sSt));
    SOX_TRY(call.input(G_tau, S * T * nn, &sG));
    SOX_TRY(call.input(w, T, &sw));
    SOX_TRY(call.output(E, 2, &oE));
    Arena ar;
    SOX_TRY(call.begin(0, &ar));
    sox::ProfScope ps(h, "gm_energies", call.stream());
    SOX_CUDA_TRY(cudaMemsetAsync(oE.out, 0, 2 * sizeof(double), call.stream()));
    sox::launch_energies(sH.in, sS.in, sg.in, sSt.in, sG.in, sw.in, p->n, p->n_tau, p->n_spin, oE.out, call.stream());
    SOX_CUDA_TRY(cudaGetLastError());
    return call.end();
  }();
  return finish(h, st);
}

int sox_mix_green(sox_handle h, long long count, double a, double *G, const double *G_new, double *change,
                  void *stream) {
  if (!h) return SOX_ERR_INVALID_ARG;
  Status st = [&]() -> Status {
    if (count < 0 || !G || !G_new || !change) return {SOX_ERR_INVALID_ARG, "bad arguments"};
    if (!(a >= 0.0 && a <= 1.0)) return {SOX_ERR_INVALID_ARG, "mixing weight must lie in [0, 1]"};
    SOX_TRY(bind_device(h));
    bool dG = false, dN = false;
    SOX_TRY(is_device_ptr(G, &dG));
    SOX_TRY(is_device_ptr(G_new, &dN));
    if (!dG || !dN) return {SOX_ERR_INVALID_ARG, "G and G_new must be device memory"};
    Call call(h, nullptr);
    Arena ar;
    SOX_TRY(call.begin(64, &ar));
    unsigned long long *chg = ar.take<unsigned long long>(1);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    SOX_CUDA_TRY(cudaMemsetAsync(chg, 0, sizeof(unsigned long long), s));
    sox::ProfScope ps(h, "mix_green", s);
    sox::launch_mix(G, G_new, count, a, chg, s);
    unsigned long long bits = 0;
    SOX_CUDA_TRY(cudaMemcpyAsync(&bits, chg, sizeof(bits), cudaMemcpyDeviceToHost, s));
    SOX_CUDA_TRY(cudaStreamSynchronize(s));
    double c;
    std::memcpy(&c, &bits, sizeof(c));
    *change = c;
    return Status::ok();
  }();
  return finish(h, st);
}

