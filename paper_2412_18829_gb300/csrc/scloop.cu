// The self-consistent loop around Sigma for molecules (Sec. II A) on the GPU: the Dyson
// equation on fermionic Matsubara frequencies (Eqs. Dyson and G0 with S = 1), the
// high-frequency tails of G, the transforms between imaginary time and frequency, the
// electron count for the chemical-potential update, the Hartree-Fock self-energy in THC
// form and the Galitskii-Migdal energies (Eqs. E1b, E2b).  FP64 throughout.
#include <algorithm>

#include "scloop.h"

namespace sox {
namespace {

using z = double2;
__device__ __forceinline__ z zmul(z a, z b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ z zfma(z a, z b, z c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

int grid_of(long long total) { return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 65535 * 4)); }

// Aug[b] = [ (i w + mu) 1 - F[s] - Sigma[s][w]  |  1 ]  for system b = s * n_w + w  (n x 2n)
__global__ void k_dyson_build(const double *omegas, double mu, const double *F, const z *Sig, int n, int n_w,
                              int n_spin, z *Aug) {
  const long long nn = (long long)n * n, total = nn * n_w * n_spin;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long b = g / nn, e = g % nn;
    const int s = (int)(b / n_w), w = (int)(b % n_w);
    const int i = (int)(e / n), j = (int)(e % n);
    z a = make_double2(-F[(long long)s * nn + e], 0.0);
    if (Sig) {
      const z sg = Sig[b * nn + e];
      a.x -= sg.x;
      a.y -= sg.y;
    }
    if (i == j) {
      a.x += mu;
      a.y += omegas[w];
    }
    z *row = Aug + b * 2 * nn + (long long)i * 2 * n;
    row[j] = a;
    row[n + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
}

// Gauss-Jordan with partial pivoting on each n x 2n system (one block per system); the
// right half becomes the inverse.  singular[0] is set for a zero pivot column.
__global__ void __launch_bounds__(256) k_gj_block(z *Aug, int n, int *singular) {
  extern __shared__ z fk[];   // column k of the system (n entries)
  __shared__ double best[256];
  __shared__ int bidx[256];
  const long long W = 2LL * n;
  z *A = Aug + (long long)blockIdx.x * n * W;
  for (int k = 0; k < n; ++k) {
    double bv = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      const z a = A[(long long)i * W + k];
      const double m2 = a.x * a.x + a.y * a.y;
      if (m2 > bv) {
        bv = m2;
        bi = i;
      }
    }
    best[threadIdx.x] = bv;
    bidx[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        const double ov = best[threadIdx.x + o];
        const int oi = bidx[threadIdx.x + o];
        if (ov > best[threadIdx.x] || (ov == best[threadIdx.x] && oi < bidx[threadIdx.x])) {
          best[threadIdx.x] = ov;
          bidx[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    if (!(best[0] > 0.0)) {
      if (threadIdx.x == 0) atomicExch(singular, 1);
      return;   // uniform: every thread sees best[0]
    }
    const int p = bidx[0];
    const z pv = A[(long long)p * W + k];
    const double d = pv.x * pv.x + pv.y * pv.y;
    const z inv = make_double2(pv.x / d, -pv.y / d);
    __syncthreads();
    for (long long j = k + threadIdx.x; j < W; j += blockDim.x) {
      const z a = A[(long long)k * W + j];
      const z b = A[(long long)p * W + j];
      if (p != k) A[(long long)p * W + j] = a;
      A[(long long)k * W + j] = zmul(b, inv);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) fk[i] = A[(long long)i * W + k];
    __syncthreads();
    const long long cols = W - (k + 1);
    for (long long e = threadIdx.x; e < (long long)n * cols; e += blockDim.x) {
      const int i = (int)(e / cols);
      if (i == k) continue;
      const long long j = k + 1 + e % cols;
      const z f = fk[i];
      z *c = A + (long long)i * W + j;
      *c = zfma(make_double2(-f.x, -f.y), A[(long long)k * W + j], *c);
    }
    __syncthreads();
  }
}

// G[b] = right half of Aug[b]
__global__ void k_right_half(const z *Aug, int n, long long batch, z *G) {
  const long long nn = (long long)n * n, total = nn * batch;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long b = g / nn, e = g % nn;
    const int i = (int)(e / n), j = (int)(e % n);
    G[g] = Aug[b * 2 * nn + (long long)i * 2 * n + n + j];
  }
}

// tails[s] = {1, A, A A + S1} with A = F - mu 1 and S1 = -(Sigma(tau_{T-1}) + Sigma(tau_0))
// (the jump of the antiperiodic Sigma(tau); zero when Sigma_tau is NULL); real [n_spin][3][n][n]
__global__ void k_tails(const double *F, double mu, const double *Sig_tau, int n, int T, int n_spin, double *tails) {
  const long long nn = (long long)n * n, total = nn * n_spin;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(g / nn);
    const long long e = g % nn;
    const int i = (int)(e / n), j = (int)(e % n);
    const double *Fs = F + (long long)s * nn;
    double a2 = 0.0;
    for (int k = 0; k < n; ++k) {
      const double aik = Fs[(long long)i * n + k] - (i == k ? mu : 0.0);
      const double akj = Fs[(long long)k * n + j] - (k == j ? mu : 0.0);
      a2 = fma(aik, akj, a2);
    }
    double s1 = 0.0;
    if (Sig_tau) {
      const double *S = Sig_tau + (long long)s * T * nn;
      s1 = -(S[(long long)(T - 1) * nn + e] + S[e]);
    }
    double *t = tails + (long long)s * 3 * nn;
    t[e] = (i == j) ? 1.0 : 0.0;
    t[nn + e] = Fs[e] - (i == j ? mu : 0.0);
    t[2 * nn + e] = a2 + s1;
  }
}

// G(tau_t) = Re[(1/beta) sum_w e^{-i w tau_t} (G(iw) - c1/(iw) - c2/(iw)^2 - c3/(iw)^3)]
//            + t1(tau) c1 + t2(tau) c2 + t3(tau) c3
// with the closed-form tau images t1 = -1/2, t2 = (2 tau - beta)/4, t3 = tau (beta - tau)/4 of the
// tails summed over all fermionic frequencies; tau on [0, beta] read as 0^+ and beta^-.
__global__ void k_iw_to_tau(const z *Giw, const double *omegas, int n_w, const double *tails, const double *tau,
                            int n_t, int n, int n_spin, double beta, double *Gtau) {
  const long long nn = (long long)n * n, total = nn * n_t * n_spin;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long e = g % nn;
    const int t = (int)((g / nn) % n_t), s = (int)(g / (nn * n_t));
    const double *c = tails + (long long)s * 3 * nn;
    const double c1 = c[e], c2 = c[nn + e], c3 = c[2 * nn + e];
    const z *G = Giw + (long long)s * n_w * nn + e;
    const double tt = tau[t];
    double acc = 0.0;
    for (int w = 0; w < n_w; ++w) {
      const double om = omegas[w];
      // residual r = G - c1/(i w) - c2/(i w)^2 - c3/(i w)^3 = G + i c1/w + c2/w^2 - i c3/w^3
      const double iw1 = 1.0 / om, iw2 = iw1 * iw1, iw3 = iw2 * iw1;
      const z gv = G[(long long)w * nn];
      const double rx = gv.x + c2 * iw2, ry = gv.y + c1 * iw1 - c3 * iw3;
      double sn, cs;
      sincos(om * tt, &sn, &cs);
      acc += rx * cs + ry * sn;   // Re[(cos - i sin)(rx + i ry)]
    }
    Gtau[g] = acc / beta - 0.5 * c1 + 0.25 * (2.0 * tt - beta) * c2 + 0.25 * tt * (beta - tt) * c3;
  }
}

// F_iw[s][w] = sum_j Tw[w][j] F_tau[s][j]  (Tw complex [n_w][n_tau], F_tau real)
__global__ void k_tau_to_iw(const z *Tw, const double *Ft, int n_w, int T, int n, int n_spin, z *Fiw) {
  const long long nn = (long long)n * n, total = nn * n_w * n_spin;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long e = g % nn;
    const int w = (int)((g / nn) % n_w), s = (int)(g / (nn * n_w));
    const double *F = Ft + (long long)s * T * nn + e;
    const z *Tr = Tw + (long long)w * T;
    z acc = make_double2(0.0, 0.0);
    for (int j = 0; j < T; ++j) {
      const double f = F[(long long)j * nn];
      acc.x = fma(Tr[j].x, f, acc.x);
      acc.y = fma(Tr[j].y, f, acc.y);
    }
    Fiw[g] = acc;
  }
}

// count[0] += sum_s Tr gamma^s, gamma = -G(beta^-)^T, from G(iw) and the tails (trace only)
__global__ void k_trace_gamma(const z *Giw, const double *omegas, int n_w, const double *tails, int n, int n_spin,
                              double beta, double *count) {
  double acc = 0.0;
  const long long nn = (long long)n * n;
  const long long total = (long long)n * n_spin;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(g / n), i = (int)(g % n);
    const long long e = (long long)i * n + i;
    const double *c = tails + (long long)s * 3 * nn;
    const double c1 = c[e], c2 = c[nn + e], c3 = c[2 * nn + e];
    const z *G = Giw + (long long)s * n_w * nn + e;
    double sum = 0.0;
    for (int w = 0; w < n_w; ++w) {
      const double om = omegas[w];
      const double iw1 = 1.0 / om, iw2 = iw1 * iw1, iw3 = iw2 * iw1;
      const z gv = G[(long long)w * nn];
      const double rx = gv.x + c2 * iw2, ry = gv.y + c1 * iw1 - c3 * iw3;
      double sn, cs;
      sincos(om * beta, &sn, &cs);
      sum += rx * cs + ry * sn;
    }
    const double gb = sum / beta - 0.5 * c1 + 0.25 * beta * c2;   // tau = beta: t3 = 0
    acc -= gb;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(count, acc);
}

// THC Hartree-Fock: d[Q] = sum_rs X[Q][r] X[Q][s] rho_rs (rho = sum_s gamma^s),
// Gam[s][P][Q] = sum_rs X[P][r] gamma^s_rs X[Q][s]
__global__ void k_hf_density(const double *X, const double *gam, int N, int n, int n_spin, double *d) {
  const long long nn = (long long)n * n;
  for (int Q = blockIdx.x * blockDim.x + threadIdx.x; Q < N; Q += gridDim.x * blockDim.x) {
    const double *x = X + (long long)Q * n;
    double acc = 0.0;
    for (int s = 0; s < n_spin; ++s)
      for (int r = 0; r < n; ++r) {
        double row = 0.0;
        for (int c = 0; c < n; ++c) row = fma(gam[s * nn + (long long)r * n + c], x[c], row);
        acc = fma(x[r], row, acc);
      }
    d[Q] = acc;
  }
}

// Sigma_HF^s[p][q] = J[p][q] - K^s[p][q] with J = sum_PQ X_Pp X_Pq V_PQ d_Q and
// K^s = sum_PQ X_Pp X_Qq V_PQ Gam^s_PQ
__global__ void k_hf_sigma(const double *X, const double *V, const double *d, const double *Gam, int N, int n,
                           int n_spin, double *S) {
  const long long nn = (long long)n * n, total = nn * n_spin;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(g / nn);
    const long long e = g % nn;
    const int p = (int)(e / n), q = (int)(e % n);
    const double *Gs = Gam + (long long)s * N * N;
    double J = 0.0, K = 0.0;
    for (int P = 0; P < N; ++P) {
      const double xp = X[(long long)P * n + p];
      double vd = 0.0, vg = 0.0;
      for (int Q = 0; Q < N; ++Q) {
        const double v = V[(long long)P * N + Q];
        vd = fma(v, d[Q], vd);
        vg = fma(v * Gs[(long long)P * N + Q], X[(long long)Q * n + q], vg);
      }
      J = fma(xp * X[(long long)P * n + q], vd, J);
      K = fma(xp, vg, K);
    }
    S[g] = J - K;
  }
}

// out[0] += sum_s sum_pq (H0 + Sigma_HF^s / 2)_pq gamma^s_pq                       (E_inf, Eq. E1b)
// out[1] -= sum_s sum_j w_j sum_pq Sigma^s_pq(tau_{T-1-j}) G^s_qp(tau_j)            (E_dyn, Eq. E2b)
__global__ void k_energies(const double *H0, const double *Shf, const double *gam, const double *Sig, const double *G,
                           const double *w, int n, int T, int n_spin, double *out) {
  const long long nn = (long long)n * n;
  double einf = 0.0, edyn = 0.0;
  const long long total1 = nn * n_spin;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total1;
       g += (long long)gridDim.x * blockDim.x) {
    const long long e = g % nn;
    einf = fma(H0[e] + 0.5 * Shf[g], gam[g], einf);
  }
  const long long total2 = nn * T * n_spin;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total2;
       g += (long long)gridDim.x * blockDim.x) {
    const long long e = g % nn;
    const int j = (int)((g / nn) % T), s = (int)(g / (nn * T));
    const int p = (int)(e / n), q = (int)(e % n);
    const double sv = Sig[((long long)s * T + (T - 1 - j)) * nn + e];
    const double gv = G[((long long)s * T + j) * nn + (long long)q * n + p];
    edyn = fma(-w[j] * sv, gv, edyn);
  }
  for (int o = 16; o > 0; o >>= 1) {
    einf += __shfl_xor_sync(0xffffffffu, einf, o);
    edyn += __shfl_xor_sync(0xffffffffu, edyn, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], einf);
    atomicAdd(&out[1], edyn);
  }
}

// G = (1 - a) G + a Gnew; change[0] = max |Gnew - G_old| (bit pattern of a non-negative double)
__global__ void k_mix(double *G, const double *Gnew, long long count, double a, unsigned long long *change) {
  double m = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const double g = G[e], gn = Gnew[e];
    m = fmax(m, fabs(gn - g));
    G[e] = (1.0 - a) * g + a * gn;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(change, (unsigned long long)__double_as_longlong(m));
}

}  // namespace

size_t dyson_bytes(int n, int n_w, int n_spin) {
  return aligned_bytes((size_t)n_spin * n_w * 2 * (size_t)n * n, 16) + 4096;
}

Status dyson(sox_handle h, int n, int n_w, int n_spin, const double *omegas, double mu, const double *F,
             const double *Sigma_iw, double *G_iw, Arena &ar, cudaStream_t s) {
  z *Aug = ar.take<z>((size_t)n_spin * n_w * 2 * (size_t)n * n);
  int *info = ar.take<int>(4);
  if (!info) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  const long long batch = (long long)n_spin * n_w;
  if (batch > 0x7fffffff) return {SOX_ERR_SHAPE, "too many Dyson systems"};
  ProfScope ps(h, "dyson", s, 3);
  SOX_CUDA_TRY(cudaMemsetAsync(info, 0, 4 * sizeof(int), s));
  k_dyson_build<<<grid_of(batch * n * n), 256, 0, s>>>(omegas, mu, F, reinterpret_cast<const z *>(Sigma_iw), n, n_w,
                                                       n_spin, Aug);
  const size_t shm = sizeof(z) * (size_t)n;
  k_gj_block<<<(unsigned)batch, 256, shm, s>>>(Aug, n, info);
  k_right_half<<<grid_of(batch * n * n), 256, 0, s>>>(Aug, n, batch, reinterpret_cast<z *>(G_iw));
  SOX_CUDA_TRY(cudaGetLastError());
  int hinfo[4] = {0, 0, 0, 0};
  SOX_CUDA_TRY(cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, s));
  SOX_CUDA_TRY(cudaStreamSynchronize(s));
  if (hinfo[0]) return {SOX_ERR_INVALID_ARG, "(i w + mu) - F - Sigma(i w) is singular at some frequency"};
  return Status::ok();
}

void launch_green_tails(const double *F, double mu, const double *Sigma_tau, int n, int T, int n_spin, double *tails,
                        cudaStream_t s) {
  k_tails<<<grid_of((long long)n * n * n_spin), 256, 0, s>>>(F, mu, Sigma_tau, n, T, n_spin, tails);
}

void launch_iw_to_tau(const double *G_iw, const double *omegas, int n_w, const double *tails, const double *tau,
                      int n_t, int n, int n_spin, double beta, double *G_tau, cudaStream_t s) {
  k_iw_to_tau<<<grid_of((long long)n * n * n_t * n_spin), 256, 0, s>>>(reinterpret_cast<const z *>(G_iw), omegas,
                                                                       n_w, tails, tau, n_t, n, n_spin, beta, G_tau);
}

void launch_tau_to_iw(const double *Tw, const double *F_tau, int n_w, int T, int n, int n_spin, double *F_iw,
                      cudaStream_t s) {
  k_tau_to_iw<<<grid_of((long long)n * n * n_w * n_spin), 256, 0, s>>>(reinterpret_cast<const z *>(Tw), F_tau, n_w, T,
                                                                       n, n_spin, reinterpret_cast<z *>(F_iw));
}

void launch_trace_gamma(const double *G_iw, const double *omegas, int n_w, const double *tails, int n, int n_spin,
                        double beta, double *count, cudaStream_t s) {
  k_trace_gamma<<<grid_of((long long)n * n_spin), 256, 0, s>>>(reinterpret_cast<const z *>(G_iw), omegas, n_w, tails,
                                                                n, n_spin, beta, count);
}

void launch_sigma_hf(const double *X, const double *V, const double *gamma, int N, int n, int n_spin, double *d,
                     double *Gam, double *S, cudaStream_t s) {
  k_hf_density<<<grid_of(N), 256, 0, s>>>(X, gamma, N, n, n_spin, d);
  for (int sp = 0; sp < n_spin; ++sp) {   // Gam[s] = X gamma^s X^T (FP64 GEMMs)
    GemmF64 a;   // T = gamma X^T -> Gam = X T; done as one GEMM pair through Gam as scratch
    a.M = N; a.Nc = n; a.K = n;
    a.A = X; a.ai = n; a.ak = 1;
    a.B = gamma + (long long)sp * n * n; a.bk = n; a.bj = 1;
    a.C = d + N + (long long)sp * N * n; a.ci = n; a.cj = 1;   // M = X gamma  (scratch after d)
    launch_gemm_f64(a, s);
    GemmF64 b;
    b.M = N; b.Nc = N; b.K = n;
    b.A = d + N + (long long)sp * N * n; b.ai = n; b.ak = 1;
    b.B = X; b.bk = 1; b.bj = n;
    b.C = Gam + (long long)sp * N * N; b.ci = N; b.cj = 1;
    launch_gemm_f64(b, s);
  }
  k_hf_sigma<<<grid_of((long long)n * n * n_spin), 256, 0, s>>>(X, V, d, Gam, N, n, n_spin, S);
}

void launch_energies(const double *H0, const double *Shf, const double *gamma, const double *Sigma_tau,
                     const double *G_tau, const double *w, int n, int T, int n_spin, double *out, cudaStream_t s) {
  k_energies<<<grid_of((long long)n * n * T * n_spin), 256, 0, s>>>(H0, Shf, gamma, Sigma_tau, G_tau, w, n, T, n_spin,
                                                                    out);
}

void launch_mix(double *G, const double *Gnew, long long count, double a, unsigned long long *change, cudaStream_t s) {
  k_mix<<<grid_of(count), 256, 0, s>>>(G, Gnew, count, a, change);
}

}  // namespace sox

namespace sox {
namespace {
// gamma[s][p][q] = -G[s][T-1][q][p]
__global__ void k_gamma_from_tau(const double *G, int n, int T, int n_spin, double *gam) {
  const long long nn = (long long)n * n, total = nn * n_spin;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(g / nn);
    const long long e = g % nn;
    const int p = (int)(e / n), q = (int)(e % n);
    gam[g] = -G[((long long)s * T + (T - 1)) * nn + (long long)q * n + p];
  }
}
}  // namespace

void launch_gamma_from_tau(const double *G_tau, int n, int T, int n_spin, double *gamma, cudaStream_t s) {
  k_gamma_from_tau<<<grid_of((long long)n * n * n_spin), 256, 0, s>>>(G_tau, n, T, n_spin, gamma);
}
}  // namespace sox
