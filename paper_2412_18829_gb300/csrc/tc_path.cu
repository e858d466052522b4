// Split-precision path of the THC-SOX chain (Sec. II C) on tcgen05 tensor cores.
//
//   mixed tensors U_Pqs = sum_Q U_PQ X_qQ X_sQ        FP32 CUDA cores, round to nearest
//                                                       (an N-long sum: the tensor core's truncating
//                                                       accumulation would cost ~1 ulp per 16 terms)
//   G_Rq, G_wP projections                              FP64 GEMM, then split per row
//   A_Pqv = sum_s U_Pqs G_sv(-tau)                      FP16x2 GEMM, split output
//   D_PR = sum_v B_PRv C_RvP (B, C never stored)        fused tcgen05 kernel
//   Sigma_tr = -sum_PR X_tR D_PR X_rP                   FP32 half-transform, FP64 final sum
#include <algorithm>
#include <string>
#include <vector>

#include "tc_kernels.h"
#include "tc_path.h"

namespace sox {
namespace {

constexpr size_t kChunkBudget = size_t(24) << 30;

inline int rup(int x, int m) { return (x + m - 1) / m * m; }

struct Geometry {
  int n, N, T, S;
  int Kp;   // n padded to 64 (K extent of the orbital contractions)
  int Np;   // N padded to 64 (K extent of the mixed-tensor GEMM)
  int NR;   // rows allocated along P / R (>= 128, rows >= N are zero)
  int RG;   // rows allocated for G(-tau)^T (>= 128)
  int Bc;   // (spin, tau) batches per chunk
  size_t fixed_bytes, per_b_bytes;
};

size_t hb(size_t count) { return aligned_bytes(count, 2); }   // FP16 buffer
size_t fb(size_t count) { return aligned_bytes(count, 4); }   // FP32 buffer
size_t db(size_t count) { return aligned_bytes(count, 8); }   // FP64 buffer

Geometry geometry(sox_handle h, int n, int N, int T, int S, bool two) {
  Geometry g{};
  g.n = n; g.N = N; g.T = T; g.S = S;
  g.Kp = rup(n, 64);
  g.Np = rup(N, 64);
  g.NR = std::max(N, 128);
  g.RG = std::max(g.Kp, 128);
  const size_t Kp2 = (size_t)g.Kp * g.Kp;
  g.fixed_bytes = fb((size_t)g.N * Kp2)                             // FP32 mixed tensor
                  + 2 * hb((size_t)g.NR * Kp2) + fb(g.N)              // U1 split
                  + 2 * hb((size_t)g.n * g.NR * g.Kp) + fb(g.N);      // U2 split
  g.per_b_bytes = 2 * db((size_t)N * n)                                // FP64 projections
                  + 4 * hb((size_t)g.NR * g.Kp) + 2 * fb(N)           // GR / GW splits
                  + 2 * hb((size_t)g.RG * g.Kp) + 2 * fb(1)           // G(-tau)^T split, scales
                  + fb(g.NR)                                          // exact per-P scale of A
                  + 2 * hb((size_t)n * g.NR * g.Kp)                   // A split
                  + 2 * fb(N)                                         // row/col factors
                  + fb((size_t)N * N) + fb((size_t)N * n) + 4096      // Dt, T
                  + fb(1);                                            // symmetry flag
  long long c = (long long)(chunk_budget(h, kChunkBudget) / std::max<size_t>(g.per_b_bytes, 1));
  c = std::max<long long>(1, std::min<long long>(c, (long long)T * S));
  g.Bc = (int)c;
  return g;
}


// Fused-kernel variant for this shape: the handle's forced choice, its cached choice, else
// (outside a stream capture, with autotuning on) each candidate is launched twice on the
// call's own data and the faster second launch wins.  The kernel is a pure function of
// its inputs, so the extra launches only cost time.
Status tune_bcd(sox_handle h, const CUtensorMap *maps, const BcdArgs &a, int grid, cudaStream_t s, int *variant) {
  const int dflt = a.Kp <= 128 ? kBcdResident : kBcdStreamed;
  if (h->variant != SOX_KERNEL_AUTO) {
    *variant = (h->variant == kBcdResident && a.Kp > 128) ? kBcdStreamed : h->variant;
    return Status::ok();
  }
  const std::string key = "bcd:" + std::to_string(a.n) + ":" + std::to_string(a.N) + ":" + std::to_string(a.batch) +
                          ":" + std::to_string(grid);
  auto it = h->tuned.find(key);
  if (it != h->tuned.end()) {
    *variant = it->second;
    return Status::ok();
  }
  *variant = dflt;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SOX_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  if (!h->autotune || cap != cudaStreamCaptureStatusNone) return Status::ok();
  const int cands[3] = {kBcdResident, kBcdStreamed, kBcdPair};
  float best = 0.f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SOX_CUDA_TRY(cudaEventCreate(&e0));
  SOX_CUDA_TRY(cudaEventCreate(&e1));
  Status st = Status::ok();
  for (int c : cands) {
    if (c == kBcdResident && a.Kp > 128) continue;
    cudaError_t e = launch_sox_bcd_tc(maps, a, grid, s, c);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_sox_bcd_tc(maps, a, grid, s, c);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      st = {SOX_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e)};
      break;
    }
    h->launches += 2;
    if (best == 0.f || ms < best) {
      best = ms;
      *variant = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st.good()) h->tuned[key] = *variant;
  return st;
}

}  // namespace

size_t tc_sigma_bytes(sox_handle h, int n, int N, int T, int S, bool two) {
  Geometry g = geometry(h, n, N, T, S, two);
  return g.fixed_bytes + g.per_b_bytes * g.Bc + 64 * 1024;
}

void tc_release(sox_handle) {}

Status tc_sigma(sox_handle h, int n, int N, int T, int S, const double *G, const double *X, const double *U1,
                const double *U2, double *Sigma, Arena &ar, cudaStream_t s) {
  const bool two = (U1 != U2);
  const Geometry g = geometry(h, n, N, T, S, two);
  const int Kp = g.Kp, NR = g.NR, RG = g.RG, Bc = g.Bc;
  const size_t Kp2 = (size_t)Kp * Kp;
  std::string err;

  // ---- fixed buffers ----
  float *Uf = ar.take<float>((size_t)N * Kp2);
  __half *U1h = ar.take<__half>((size_t)NR * Kp2), *U1l = ar.take<__half>((size_t)NR * Kp2);
  float *inv_u1 = ar.take<float>(N);
  __half *U2h = ar.take<__half>((size_t)n * NR * Kp), *U2l = ar.take<__half>((size_t)n * NR * Kp);
  float *inv_u2 = ar.take<float>(N);
  // ---- per-chunk buffers ----
  double *GR64 = ar.take<double>((size_t)Bc * N * n), *GW64 = ar.take<double>((size_t)Bc * N * n);
  __half *GRh = ar.take<__half>((size_t)Bc * NR * Kp), *GRl = ar.take<__half>((size_t)Bc * NR * Kp);
  __half *GWh = ar.take<__half>((size_t)Bc * NR * Kp), *GWl = ar.take<__half>((size_t)Bc * NR * Kp);
  float *inv_gr = ar.take<float>((size_t)Bc * N), *inv_gw = ar.take<float>((size_t)Bc * N);
  __half *Gmh = ar.take<__half>((size_t)Bc * RG * Kp), *Gml = ar.take<__half>((size_t)Bc * RG * Kp);
  float *gsc = ar.take<float>(Bc), *osc = ar.take<float>(Bc);
  float *asc = ar.take<float>((size_t)Bc * NR);
  __half *Ah = ar.take<__half>((size_t)Bc * n * NR * Kp), *Al = ar.take<__half>((size_t)Bc * n * NR * Kp);
  float *rowf = ar.take<float>((size_t)Bc * N), *colf = ar.take<float>((size_t)Bc * N);
  float *Dt = ar.take<float>((size_t)Bc * N * N);
  float *Tm = ar.take<float>((size_t)Bc * N * n);
  int *symf = ar.take<int>((size_t)Bc);
  if (!symf) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};

  const long long limit = h->spin_limit;
  auto grid_for = [&](long long tiles) { return (int)std::max<long long>(1, std::min<long long>(tiles, h->sm_count)); };

  // ---- mixed tensors (Eq. U_contraction at k = 0) ----
  {
    ProfScope ps(h, "mixed_f32", s, two ? 4 : 2);
    SOX_CUDA_TRY(cudaMemsetAsync(U1h, 0, hb((size_t)NR * Kp2), s));
    SOX_CUDA_TRY(cudaMemsetAsync(U1l, 0, hb((size_t)NR * Kp2), s));
    SOX_CUDA_TRY(cudaMemsetAsync(U2h, 0, hb((size_t)n * NR * Kp), s));
    SOX_CUDA_TRY(cudaMemsetAsync(U2l, 0, hb((size_t)n * NR * Kp), s));
    const double *src[2] = {U1, U2};
    for (int k = 0; k < (two ? 2 : 1); ++k) {
      launch_mixed_f32(src[k], X, N, n, Kp, Uf, s);
      const bool slot1 = (k == 0), slot2 = two ? (k == 1) : true;
      launch_split_mixed(Uf, N, NR, n, Kp, slot1 ? U1h : nullptr, slot1 ? U1l : nullptr, slot2 ? U2h : nullptr,
                         slot2 ? U2l : nullptr, slot1 ? inv_u1 : inv_u2, s);
      if (!two) SOX_CUDA_TRY(cudaMemcpyAsync(inv_u2, inv_u1, 4 * (size_t)N, cudaMemcpyDeviceToDevice, s));
    }
  }

  // ---- tensor maps of the per-chunk buffers (fixed addresses, reused per chunk) ----
  CUtensorMap bcd[12], agemm[6];
  if (!make_tmap_f16_3d(&bcd[0], Ah, Kp, NR, (uint64_t)Bc * n, 64, 128, &err) ||
      !make_tmap_f16_3d(&bcd[1], Al, Kp, NR, (uint64_t)Bc * n, 64, 128, &err) ||
      !make_tmap_f16_3d(&bcd[2], GRh, Kp, NR, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&bcd[3], GRl, Kp, NR, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&bcd[4], GWh, Kp, NR, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&bcd[5], GWl, Kp, NR, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&bcd[6], U2h, Kp, NR, n, 64, 128, &err) ||
      !make_tmap_f16_3d(&bcd[7], U2l, Kp, NR, n, 64, 128, &err) ||
      !make_tmap_f16_3d(&bcd[8], GRh, Kp, NR, Bc, 64, 64, &err) ||
      !make_tmap_f16_3d(&bcd[9], GRl, Kp, NR, Bc, 64, 64, &err) ||
      !make_tmap_f16_3d(&bcd[10], U2h, Kp, NR, n, 64, 64, &err) ||
      !make_tmap_f16_3d(&bcd[11], U2l, Kp, NR, n, 64, 64, &err) ||
      !make_tmap_f16_3d(&agemm[0], Gmh, Kp, RG, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&agemm[1], Gml, Kp, RG, Bc, 64, 128, &err) ||
      !make_tmap_f16_3d(&agemm[2], U1h, Kp, (uint64_t)NR * Kp, 1, 64, 128, &err) ||
      !make_tmap_f16_3d(&agemm[3], U1l, Kp, (uint64_t)NR * Kp, 1, 64, 128, &err) ||
      !make_tmap_f16_store4d(&agemm[4], Ah, Kp, NR, n, Bc, &err) ||
      !make_tmap_f16_store4d(&agemm[5], Al, Kp, NR, n, Bc, &err))
    return {SOX_ERR_CUDA, err};

  const bool exact_a = (Kp <= 128);
  const int B = S * T;
  for (int b0 = 0; b0 < B; b0 += Bc) {
    const int bc = std::min(Bc, B - b0);
    const double *Gc = G + (long long)b0 * n * n;
    {  // FP64 projections G_Rq = X G, G_wP^T = X G^T, then row splits.  For a symmetric
       // G(tau) (real molecular orbitals) G_wP^T = G_Rq: a device flag per (spin, tau)
       // lets the second GEMM skip its blocks and the split read G_Rq instead.
      ProfScope ps(h, "project_f64", s, 5);
      launch_symmetry_flags(Gc, n, bc, symf, s);
      GemmF64 gp;
      gp.M = N; gp.Nc = n; gp.K = n; gp.batch = bc;
      gp.A = X; gp.ai = n; gp.ak = 1;
      gp.B = Gc; gp.sB = (long long)n * n; gp.bk = n; gp.bj = 1;
      gp.C = GR64; gp.sC = (long long)N * n; gp.ci = n; gp.cj = 1;
      launch_gemm_f64(gp, s);
      GemmF64 gw = gp;
      gw.bk = 1; gw.bj = n;
      gw.C = GW64;
      gw.skip = symf;
      launch_gemm_f64(gw, s);
      launch_split_rows_f64(GR64, n, (long long)N * n, N, NR, n, Kp, GRh, GRl, inv_gr, bc, s);
      launch_split_rows_f64(GW64, n, (long long)N * n, N, NR, n, Kp, GWh, GWl, inv_gw, bc, s, GR64, symf);
    }
    {  // A_Pqv = sum_s G(-tau)_sv U_Pqs
      ProfScope ps(h, "A_tc", s, 2);
      launch_prep_gminus(G, n, T, bc, Kp, Gmh, Gml, gsc, osc, b0, RG, s);
      GemmTcArgs ga;
      ga.M = n; ga.Ncols = NR * Kp; ga.Kp = Kp; ga.K = n; ga.batch = bc;
      ga.batchA_shared = 0; ga.batchB_shared = 1;
      // n <= 128: one tile holds all (v, q) of each P -> exact per-P scale; else the a-priori bound
      ga.mode = exact_a ? kStoreSplitGroup : kStoreSplit;
      ga.out_scale = osc;
      ga.group = Kp; ga.n_groups = NR; ga.group_scale = asc;
      ga.spin_limit = limit; ga.status = h->d_status;
      const long long tiles = (long long)bc * ((n + 127) / 128) * ((NR * Kp + 127) / 128);
      SOX_CUDA_TRY(launch_gemm_f16x2(agemm, ga, grid_for(tiles), s));
    }
    launch_bcd_scales(inv_u1, gsc, osc, exact_a ? asc : nullptr, NR, inv_gw, inv_gr, inv_u2, N, bc, rowf, colf, s);
    h->launches += 1;
    {  // fused B / C / Hadamard-reduce
      ProfScope ps(h, "sox_bcd_tc", s);
      BcdArgs ba;
      ba.n = n; ba.N = N; ba.Kp = Kp; ba.batch = bc;
      v_range(h, n, &ba.v0, &ba.v1);
      ba.spin_limit = limit; ba.status = h->d_status;
      ba.row_scale = rowf; ba.col_scale = colf;
      ba.Dt = Dt; ba.ldD = N;
      const int tP = (N + 127) / 128;
      const int grid = grid_for((long long)bc * tP * tP);
      int variant = 0;
      SOX_TRY(tune_bcd(h, bcd, ba, grid, s, &variant));
      SOX_CUDA_TRY(launch_sox_bcd_tc(bcd, ba, grid, s, variant));
    }
    {  // back-projection to orbitals
      ProfScope ps(h, "backproject", s, 2);
      launch_backproject_T(Dt, N, X, N, n, bc, Tm, s);
      // bare SOX with a symmetric G(tau) has a symmetric Sigma(tau)
      // (a partial v range breaks that symmetry: then every block is computed)
      launch_backproject_sigma(X, Tm, N, n, bc, Sigma + (long long)b0 * n * n, (long long)n * n, s,
                               (two || !v_range_is_full(h, n)) ? nullptr : symf);
    }
  }
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

// ---------------------------------------------------------------------------------------
// The uneven batch (bare SOX of several molecules of different sizes): every instance's
// chain up to A and after D runs per instance, and the fused B / C / Hadamard step of one tau
// chunk of every instance runs as one persistent launch (k_sox_bcd_multi).  Instances share
// the number of tau chunks; each chunk holds ceil(B_i / nc) of instance i's batches.
// ---------------------------------------------------------------------------------------
namespace {

struct BatchGeo {
  int nc = 1;
  std::vector<int> Bc;
  size_t bytes = 0;
};

constexpr size_t kBatchBudget = size_t(128) << 30;

// Per-instance chunk sizes: every instance starts whole (all its (spin, tau) batches in one
// chunk); while the batch's buffers exceed the budget, the instance holding the most chunk
// memory halves its chunk.  Small instances thus finish in the first chunk with large
// launches of their own, and only the large ones are spread over further chunks.
BatchGeo batch_geometry(sox_handle h, int count, const int *n, const int *N, const int *T, const int *S) {
  BatchGeo bg;
  const size_t budget = chunk_budget(h, kBatchBudget);
  std::vector<Geometry> g(count);
  std::vector<long long> B(count);
  bg.Bc.assign(count, 1);
  size_t fixed = 0;
  for (int i = 0; i < count; ++i) {
    g[i] = geometry(nullptr, n[i], N[i], T[i], S[i], false);
    B[i] = (long long)T[i] * S[i];
    bg.Bc[i] = (int)B[i];
    fixed += g[i].fixed_bytes + 64 * 1024;
  }
  auto chunk_mem = [&](int i) { return g[i].per_b_bytes * (size_t)bg.Bc[i]; };
  for (;;) {
    size_t total = fixed;
    int hog = -1;
    for (int i = 0; i < count; ++i) {
      total += chunk_mem(i);
      if (bg.Bc[i] > 1 && (hog < 0 || chunk_mem(i) > chunk_mem(hog))) hog = i;
    }
    if (total <= budget || hog < 0) {
      bg.bytes = total;
      break;
    }
    bg.Bc[hog] = (bg.Bc[hog] + 1) / 2;
  }
  bg.nc = 1;
  for (int i = 0; i < count; ++i) bg.nc = std::max<int>(bg.nc, (int)((B[i] + bg.Bc[i] - 1) / bg.Bc[i]));
  return bg;
}

struct Inst {
  int n, N, T, S, Kp, NR, RG, Bc;
  const double *G, *X, *V;
  double *Sigma;
  float *Uf, *inv_u1, *inv_u2;
  __half *U1h, *U1l, *U2h, *U2l;
  double *GR64, *GW64;
  __half *GRh, *GRl, *GWh, *GWl, *Gmh, *Gml, *Ah, *Al;
  float *inv_gr, *inv_gw, *gsc, *osc, *asc, *rowf, *colf, *Dt, *Tm;
  int *symf;
  CUtensorMap bcd[8], agemm[6];
};

}  // namespace

size_t tc_sigma_batch_bytes(sox_handle h, int count, const int *n, const int *N, const int *T, const int *S) {
  return batch_geometry(h, count, n, N, T, S).bytes + 64 * 1024;
}

Status tc_sigma_batch(sox_handle h, int count, const int *n, const int *N, const int *T, const int *S,
                      const double *const *G, const double *const *X, const double *const *V, double *const *Sigma,
                      Arena &ar, cudaStream_t s) {
  if (count <= 0) return Status::ok();
  const BatchGeo bg = batch_geometry(h, count, n, N, T, S);
  std::vector<Inst> in(count);
  std::string err;
  for (int i = 0; i < count; ++i) {
    Inst &c = in[i];
    const Geometry g = geometry(nullptr, n[i], N[i], T[i], S[i], false);
    c.n = n[i]; c.N = N[i]; c.T = T[i]; c.S = S[i];
    c.Kp = g.Kp; c.NR = g.NR; c.RG = g.RG; c.Bc = bg.Bc[i];
    c.G = G[i]; c.X = X[i]; c.V = V[i]; c.Sigma = Sigma[i];
    const int nn = c.n, NN = c.N, Kp = c.Kp, NR = c.NR, RG = c.RG, Bc = c.Bc;
    const size_t Kp2 = (size_t)Kp * Kp;
    c.Uf = ar.take<float>((size_t)NN * Kp2);
    c.U1h = ar.take<__half>((size_t)NR * Kp2); c.U1l = ar.take<__half>((size_t)NR * Kp2);
    c.inv_u1 = ar.take<float>(NN);
    c.U2h = ar.take<__half>((size_t)nn * NR * Kp); c.U2l = ar.take<__half>((size_t)nn * NR * Kp);
    c.inv_u2 = ar.take<float>(NN);
    c.GR64 = ar.take<double>((size_t)Bc * NN * nn); c.GW64 = ar.take<double>((size_t)Bc * NN * nn);
    c.GRh = ar.take<__half>((size_t)Bc * NR * Kp); c.GRl = ar.take<__half>((size_t)Bc * NR * Kp);
    c.GWh = ar.take<__half>((size_t)Bc * NR * Kp); c.GWl = ar.take<__half>((size_t)Bc * NR * Kp);
    c.inv_gr = ar.take<float>((size_t)Bc * NN); c.inv_gw = ar.take<float>((size_t)Bc * NN);
    c.Gmh = ar.take<__half>((size_t)Bc * RG * Kp); c.Gml = ar.take<__half>((size_t)Bc * RG * Kp);
    c.gsc = ar.take<float>(Bc); c.osc = ar.take<float>(Bc);
    c.asc = ar.take<float>((size_t)Bc * NR);
    c.Ah = ar.take<__half>((size_t)Bc * nn * NR * Kp); c.Al = ar.take<__half>((size_t)Bc * nn * NR * Kp);
    c.rowf = ar.take<float>((size_t)Bc * NN); c.colf = ar.take<float>((size_t)Bc * NN);
    c.Dt = ar.take<float>((size_t)Bc * NN * NN);
    c.Tm = ar.take<float>((size_t)Bc * NN * nn);
    c.symf = ar.take<int>((size_t)Bc);
    if (!c.symf) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
    if (!make_tmap_f16_3d(&c.bcd[0], c.Ah, Kp, NR, (uint64_t)Bc * nn, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[1], c.Al, Kp, NR, (uint64_t)Bc * nn, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[2], c.GRh, Kp, NR, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[3], c.GRl, Kp, NR, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[4], c.GWh, Kp, NR, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[5], c.GWl, Kp, NR, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[6], c.U2h, Kp, NR, nn, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[7], c.U2l, Kp, NR, nn, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.agemm[0], c.Gmh, Kp, RG, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.agemm[1], c.Gml, Kp, RG, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.agemm[2], c.U1h, Kp, (uint64_t)NR * Kp, 1, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.agemm[3], c.U1l, Kp, (uint64_t)NR * Kp, 1, 64, 128, &err) ||
        !make_tmap_f16_store4d(&c.agemm[4], c.Ah, Kp, NR, nn, Bc, &err) ||
        !make_tmap_f16_store4d(&c.agemm[5], c.Al, Kp, NR, nn, Bc, &err))
      return {SOX_ERR_CUDA, "batch maps: " + err};
  }
  const long long limit = h->spin_limit;
  auto grid_for = [&](long long tiles) { return (int)std::max<long long>(1, std::min<long long>(tiles, h->sm_count)); };
  // mixed tensors of every instance (Eq. U_contraction at k = 0; one interaction in both slots)
  {
    ProfScope ps(h, "mixed_f32", s, 2 * count);
    for (Inst &c : in) {
      const size_t Kp2 = (size_t)c.Kp * c.Kp;
      SOX_CUDA_TRY(cudaMemsetAsync(c.U1h, 0, hb((size_t)c.NR * Kp2), s));
      SOX_CUDA_TRY(cudaMemsetAsync(c.U1l, 0, hb((size_t)c.NR * Kp2), s));
      SOX_CUDA_TRY(cudaMemsetAsync(c.U2h, 0, hb((size_t)c.n * c.NR * c.Kp), s));
      SOX_CUDA_TRY(cudaMemsetAsync(c.U2l, 0, hb((size_t)c.n * c.NR * c.Kp), s));
      launch_mixed_f32(c.V, c.X, c.N, c.n, c.Kp, c.Uf, s);
      launch_split_mixed(c.Uf, c.N, c.NR, c.n, c.Kp, c.U1h, c.U1l, c.U2h, c.U2l, c.inv_u1, s);
      SOX_CUDA_TRY(cudaMemcpyAsync(c.inv_u2, c.inv_u1, 4 * (size_t)c.N, cudaMemcpyDeviceToDevice, s));
    }
  }
  // instances by cost per tile (n Kp), largest first: the persistent grid ends on cheap tiles
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (long long)in[x].n * in[x].Kp > (long long)in[y].n * in[y].Kp;
  });
  for (int k = 0; k < bg.nc; ++k) {
    // ---- per instance: FP64 projections, row splits, A, the B/C scales ----
    for (Inst &c : in) {
      const int B = c.S * c.T, b0 = k * c.Bc, bc = std::min(c.Bc, B - b0);
      if (bc <= 0) continue;
      const double *Gc = c.G + (long long)b0 * c.n * c.n;
      {
        ProfScope ps(h, "project_f64", s, 5);
        launch_symmetry_flags(Gc, c.n, bc, c.symf, s);
        GemmF64 gp;
        gp.M = c.N; gp.Nc = c.n; gp.K = c.n; gp.batch = bc;
        gp.A = c.X; gp.ai = c.n; gp.ak = 1;
        gp.B = Gc; gp.sB = (long long)c.n * c.n; gp.bk = c.n; gp.bj = 1;
        gp.C = c.GR64; gp.sC = (long long)c.N * c.n; gp.ci = c.n; gp.cj = 1;
        launch_gemm_f64(gp, s);
        GemmF64 gw = gp;
        gw.bk = 1; gw.bj = c.n;
        gw.C = c.GW64;
        gw.skip = c.symf;
        launch_gemm_f64(gw, s);
        launch_split_rows_f64(c.GR64, c.n, (long long)c.N * c.n, c.N, c.NR, c.n, c.Kp, c.GRh, c.GRl, c.inv_gr, bc, s);
        launch_split_rows_f64(c.GW64, c.n, (long long)c.N * c.n, c.N, c.NR, c.n, c.Kp, c.GWh, c.GWl, c.inv_gw, bc, s,
                              c.GR64, c.symf);
      }
      {
        ProfScope ps(h, "A_tc", s, 2);
        const bool exact_a = (c.Kp <= 128);
        launch_prep_gminus(c.G, c.n, c.T, bc, c.Kp, c.Gmh, c.Gml, c.gsc, c.osc, b0, c.RG, s);
        GemmTcArgs ga;
        ga.M = c.n; ga.Ncols = c.NR * c.Kp; ga.Kp = c.Kp; ga.K = c.n; ga.batch = bc;
        ga.batchA_shared = 0; ga.batchB_shared = 1;
        ga.mode = exact_a ? kStoreSplitGroup : kStoreSplit;
        ga.out_scale = c.osc;
        ga.group = c.Kp; ga.n_groups = c.NR; ga.group_scale = c.asc;
        ga.spin_limit = limit; ga.status = h->d_status;
        const long long tiles = (long long)bc * ((c.n + 127) / 128) * (((long long)c.NR * c.Kp + 127) / 128);
        SOX_CUDA_TRY(launch_gemm_f16x2(c.agemm, ga, grid_for(tiles), s));
        launch_bcd_scales(c.inv_u1, c.gsc, c.osc, exact_a ? c.asc : nullptr, c.NR, c.inv_gw, c.inv_gr, c.inv_u2, c.N,
                          bc, c.rowf, c.colf, s);
        h->launches += 1;
      }
    }
    // ---- one persistent fused launch over the chunk's tiles of every instance ----
    {
      ProfScope ps(h, "sox_bcd_tc", s, 0);
      BcdJobs jobs;
      jobs.spin_limit = limit;
      jobs.status = h->d_status;
      auto flush = [&]() -> Status {
        if (jobs.count == 0) return Status::ok();
        h->launches += 1;
        SOX_CUDA_TRY(launch_sox_bcd_multi(jobs, grid_for(jobs.total), s));
        jobs.count = 0;
        jobs.total = 0;
        return Status::ok();
      };
      for (int oi : order) {
        Inst &c = in[oi];
        const int B = c.S * c.T, b0 = k * c.Bc, bc = std::min(c.Bc, B - b0);
        if (bc <= 0) continue;
        if (jobs.count == kMaxBcdJobs) SOX_TRY(flush());
        BcdJob &J = jobs.job[jobs.count++];
        for (int m = 0; m < 8; ++m) J.maps[m] = c.bcd[m];
        J.n = c.n; J.N = c.N; J.Kp = c.Kp; J.batch = bc;
        v_range(h, c.n, &J.v0, &J.v1);
        J.v1 = (J.v1 <= 0 || J.v1 > c.n) ? c.n : J.v1;
        J.v0 = J.v0 < 0 ? 0 : std::min(J.v0, J.v1);
        J.row_scale = c.rowf; J.col_scale = c.colf;
        J.Dt = c.Dt; J.ldD = c.N;
        J.unit0 = jobs.total;
        const long long tP = (c.N + 127) / 128;
        jobs.total += (long long)bc * tP * tP;
      }
      SOX_TRY(flush());
    }
    // ---- per instance: back-projection to orbitals ----
    for (Inst &c : in) {
      const int B = c.S * c.T, b0 = k * c.Bc, bc = std::min(c.Bc, B - b0);
      if (bc <= 0) continue;
      ProfScope ps(h, "backproject", s, 2);
      launch_backproject_T(c.Dt, c.N, c.X, c.N, c.n, bc, c.Tm, s);
      launch_backproject_sigma(c.X, c.Tm, c.N, c.n, bc, c.Sigma + (long long)b0 * c.n * c.n, (long long)c.n * c.n, s,
                               v_range_is_full(h, c.n) ? c.symf : nullptr);
    }
  }
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

}  // namespace sox
