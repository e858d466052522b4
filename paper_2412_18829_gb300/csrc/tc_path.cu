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

#include "tc_kernels.h"
#include "tc_path.h"

namespace sox {
namespace {

constexpr size_t kChunkBudget = size_t(24) << 30;
// The (spin, tau) batches are processed in at least this many chunks (when there are that
// many), two buffer sets in turn: chunk k+1's FP64 projections and chunk k-1's back-projection
// run on a second stream while chunk k's fused kernel holds the tensor cores.
constexpr int kPipeChunks = 4;

inline int rup(int x, int m) { return (x + m - 1) / m * m; }

struct Geometry {
  int n, N, T, S;
  int Kp;    // n padded to 64 (K extent of the orbital contractions)
  int Np;    // N padded to 64 (K extent of the mixed-tensor GEMM)
  int NR;    // rows allocated along P / R (>= 128, rows >= N are zero)
  int RG;    // rows allocated for G(-tau)^T (>= 128)
  int Bc;    // (spin, tau) batches per chunk
  int sets;  // buffer sets (2: pipelined chunks)
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
  const long long B = (long long)T * S;
  const size_t per = std::max<size_t>(g.per_b_bytes, 1);
  const size_t budget = chunk_budget(h, kChunkBudget);
  if (B >= 2) {
    const long long c2 = std::max<long long>(1, (long long)(budget / (2 * per)));
    const long long nc = std::max<long long>((B + c2 - 1) / c2, std::min<long long>(kPipeChunks, B));
    g.Bc = (int)((B + nc - 1) / nc);
    g.sets = 2;
  } else {
    g.Bc = 1;
    g.sets = 1;
  }
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
  return g.fixed_bytes + g.per_b_bytes * g.Bc * g.sets + 64 * 1024;
}

void tc_release(sox_handle h) {
  for (cudaEvent_t &e : h->pipe_ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  if (h->side) {
    cudaStreamDestroy(h->side);
    h->side = nullptr;
  }
}

// The second stream and the events of the chunk pipeline, created once per handle (at
// handle creation for split-precision handles, so that no call inside a stream capture
// creates them).
Status tc_prepare(sox_handle h) {
  if (h->side) return Status::ok();
  int least = 0, greatest = 0;
  SOX_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  h->prio_high = greatest;
  for (cudaEvent_t &e : h->pipe_ev) SOX_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  SOX_CUDA_TRY(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, least));
  return Status::ok();
}

namespace {

// Per-chunk buffers of one set.
struct ChunkBufs {
  double *GR64, *GW64;
  __half *GRh, *GRl, *GWh, *GWl, *Gmh, *Gml, *Ah, *Al;
  float *inv_gr, *inv_gw, *gsc, *osc, *asc, *rowf, *colf, *Dt, *Tm;
  int *symf;
  CUtensorMap bcd[12], agemm[6];
};

}  // namespace

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
  // ---- per-chunk buffers (one set per chunk in flight) ----
  ChunkBufs cb[2];
  for (int k = 0; k < g.sets; ++k) {
    ChunkBufs &c = cb[k];
    c.GR64 = ar.take<double>((size_t)Bc * N * n);
    c.GW64 = ar.take<double>((size_t)Bc * N * n);
    c.GRh = ar.take<__half>((size_t)Bc * NR * Kp); c.GRl = ar.take<__half>((size_t)Bc * NR * Kp);
    c.GWh = ar.take<__half>((size_t)Bc * NR * Kp); c.GWl = ar.take<__half>((size_t)Bc * NR * Kp);
    c.inv_gr = ar.take<float>((size_t)Bc * N); c.inv_gw = ar.take<float>((size_t)Bc * N);
    c.Gmh = ar.take<__half>((size_t)Bc * RG * Kp); c.Gml = ar.take<__half>((size_t)Bc * RG * Kp);
    c.gsc = ar.take<float>(Bc); c.osc = ar.take<float>(Bc);
    c.asc = ar.take<float>((size_t)Bc * NR);
    c.Ah = ar.take<__half>((size_t)Bc * n * NR * Kp); c.Al = ar.take<__half>((size_t)Bc * n * NR * Kp);
    c.rowf = ar.take<float>((size_t)Bc * N); c.colf = ar.take<float>((size_t)Bc * N);
    c.Dt = ar.take<float>((size_t)Bc * N * N);
    c.Tm = ar.take<float>((size_t)Bc * N * n);
    c.symf = ar.take<int>((size_t)Bc);
    if (!c.symf) return {SOX_ERR_OOM, "workspace too small (internal sizing error)"};
  }

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
  for (int k = 0; k < g.sets; ++k) {
    ChunkBufs &c = cb[k];
    if (!make_tmap_f16_3d(&c.bcd[0], c.Ah, Kp, NR, (uint64_t)Bc * n, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[1], c.Al, Kp, NR, (uint64_t)Bc * n, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[2], c.GRh, Kp, NR, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[3], c.GRl, Kp, NR, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[4], c.GWh, Kp, NR, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[5], c.GWl, Kp, NR, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[6], U2h, Kp, NR, n, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[7], U2l, Kp, NR, n, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.bcd[8], c.GRh, Kp, NR, Bc, 64, 64, &err) ||
        !make_tmap_f16_3d(&c.bcd[9], c.GRl, Kp, NR, Bc, 64, 64, &err) ||
        !make_tmap_f16_3d(&c.bcd[10], U2h, Kp, NR, n, 64, 64, &err) ||
        !make_tmap_f16_3d(&c.bcd[11], U2l, Kp, NR, n, 64, 64, &err) ||
        !make_tmap_f16_3d(&c.agemm[0], c.Gmh, Kp, RG, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.agemm[1], c.Gml, Kp, RG, Bc, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.agemm[2], U1h, Kp, (uint64_t)NR * Kp, 1, 64, 128, &err) ||
        !make_tmap_f16_3d(&c.agemm[3], U1l, Kp, (uint64_t)NR * Kp, 1, 64, 128, &err) ||
        !make_tmap_f16_store4d(&c.agemm[4], c.Ah, Kp, NR, n, Bc, &err) ||
        !make_tmap_f16_store4d(&c.agemm[5], c.Al, Kp, NR, n, Bc, &err))
      return {SOX_ERR_CUDA, err};
  }

  const bool exact_a = (Kp <= 128);
  const int B = S * T;
  const int nc = (B + Bc - 1) / Bc;
  // bare SOX with a symmetric G(tau) has a symmetric Sigma(tau) (a partial v range breaks
  // that symmetry: then every block is computed)
  const bool sym_sigma = !two && v_range_is_full(h, n);

  // FP64 projections G_Rq = X G, G_wP^T = X G^T of chunk k, then row splits.  For a symmetric
  // G(tau) (real molecular orbitals) G_wP^T = G_Rq: a device flag per (spin, tau) lets the
  // second GEMM skip its blocks and the split read G_Rq instead.  FP64 GEMMs in blocks that
  // fit beside a fused CTA when they run on the second stream.
  auto project = [&](int k, cudaStream_t st) -> Status {
    const int b0 = k * Bc, bc = std::min(Bc, B - b0);
    const ChunkBufs &c = cb[k % g.sets];
    const double *Gc = G + (long long)b0 * n * n;
    ProfScope ps(h, "project_f64", st, 5);
    launch_symmetry_flags(Gc, n, bc, c.symf, st);
    GemmF64 gp;
    gp.M = N; gp.Nc = n; gp.K = n; gp.batch = bc;
    gp.A = X; gp.ai = n; gp.ak = 1;
    gp.B = Gc; gp.sB = (long long)n * n; gp.bk = n; gp.bj = 1;
    gp.C = c.GR64; gp.sC = (long long)N * n; gp.ci = n; gp.cj = 1;
    GemmF64 gw = gp;
    gw.bk = 1; gw.bj = n;
    gw.C = c.GW64;
    gw.skip = c.symf;
    if (g.sets > 1) {
      launch_gemm_f64_lite(gp, st);
      launch_gemm_f64_lite(gw, st);
    } else {
      launch_gemm_f64(gp, st);
      launch_gemm_f64(gw, st);
    }
    launch_split_rows_f64(c.GR64, n, (long long)N * n, N, NR, n, Kp, c.GRh, c.GRl, c.inv_gr, bc, st);
    launch_split_rows_f64(c.GW64, n, (long long)N * n, N, NR, n, Kp, c.GWh, c.GWl, c.inv_gw, bc, st, c.GR64, c.symf);
    return Status::ok();
  };
  // Sigma_tr = -sum_PR X_tR D_PR X_rP of chunk k: FP32 half-transform, FP64 final sum
  auto backproject = [&](int k, cudaStream_t st) {
    const int b0 = k * Bc, bc = std::min(Bc, B - b0);
    const ChunkBufs &c = cb[k % g.sets];
    ProfScope ps(h, "backproject", st, 2);
    launch_backproject_T(c.Dt, N, X, N, n, bc, c.Tm, st);
    launch_backproject_sigma(X, c.Tm, N, n, bc, Sigma + (long long)b0 * n * n, (long long)n * n, st,
                             sym_sigma ? c.symf : nullptr);
  };
  // A_Pqv = sum_s G(-tau)_sv U_Pqs, the B/C scales and the fused B / C / Hadamard-reduce
  auto tensor_steps = [&](int k, cudaStream_t st, int prio) -> Status {
    const int b0 = k * Bc, bc = std::min(Bc, B - b0);
    ChunkBufs &c = cb[k % g.sets];
    {
      ProfScope ps(h, "A_tc", st, 2);
      launch_prep_gminus(G, n, T, bc, Kp, c.Gmh, c.Gml, c.gsc, c.osc, b0, RG, st);
      GemmTcArgs ga;
      ga.M = n; ga.Ncols = NR * Kp; ga.Kp = Kp; ga.K = n; ga.batch = bc;
      ga.batchA_shared = 0; ga.batchB_shared = 1;
      // n <= 128: one tile holds all (v, q) of each P -> exact per-P scale; else the a-priori bound
      ga.mode = exact_a ? kStoreSplitGroup : kStoreSplit;
      ga.out_scale = c.osc;
      ga.group = Kp; ga.n_groups = NR; ga.group_scale = c.asc;
      ga.spin_limit = limit; ga.status = h->d_status;
      const long long tiles = (long long)bc * ((n + 127) / 128) * ((NR * Kp + 127) / 128);
      SOX_CUDA_TRY(launch_gemm_f16x2(c.agemm, ga, grid_for(tiles), st));
    }
    launch_bcd_scales(inv_u1, c.gsc, c.osc, exact_a ? c.asc : nullptr, NR, c.inv_gw, c.inv_gr, inv_u2, N, bc, c.rowf,
                      c.colf, st);
    h->launches += 1;
    ProfScope ps(h, "sox_bcd_tc", st);
    BcdArgs ba;
    ba.n = n; ba.N = N; ba.Kp = Kp; ba.batch = bc;
    v_range(h, n, &ba.v0, &ba.v1);
    ba.spin_limit = limit; ba.status = h->d_status;
    ba.row_scale = c.rowf; ba.col_scale = c.colf;
    ba.Dt = c.Dt; ba.ldD = N;
    const int tP = (N + 127) / 128;
    const int grid = grid_for((long long)bc * tP * tP);
    int variant = 0;
    SOX_TRY(tune_bcd(h, c.bcd, ba, grid, st, &variant));
    SOX_CUDA_TRY(launch_sox_bcd_tc(c.bcd, ba, grid, st, variant, prio));
    return Status::ok();
  };

  if (g.sets == 1 || nc == 1) {
    for (int k = 0; k < nc; ++k) {
      SOX_TRY(project(k, s));
      SOX_TRY(tensor_steps(k, s, 0));
      backproject(k, s);
    }
    SOX_CUDA_TRY(cudaGetLastError());
    return Status::ok();
  }

  // ---- pipelined chunks: s runs the tensor-core steps, the side stream the FP64 ends ----
  //   side: proj(0) proj(1) | back(0) proj(2) | back(1) proj(3) | ... | back(nc-1)
  //   s:    [mixed] A+fused(0) | A+fused(1) | ...
  // Set k % 2 is rewritten by proj(k + 2) only after back(k) (same stream), which itself waits
  // for fused(k); fused(k + 2) waits for proj(k + 2).  The fused kernels launch at the
  // device's greatest priority so their CTAs take SMs ahead of pending FP64 blocks.
  SOX_TRY(tc_prepare(h));
  cudaStream_t side = h->side;
  cudaEvent_t ev_fork = h->pipe_ev[0], ev_join = h->pipe_ev[1];
  cudaEvent_t ev_proj[2] = {h->pipe_ev[2], h->pipe_ev[3]}, ev_fused[2] = {h->pipe_ev[4], h->pipe_ev[5]};
  SOX_CUDA_TRY(cudaEventRecord(ev_fork, s));
  SOX_CUDA_TRY(cudaStreamWaitEvent(side, ev_fork, 0));
  for (int k = 0; k < std::min(nc, 2); ++k) {
    SOX_TRY(project(k, side));
    SOX_CUDA_TRY(cudaEventRecord(ev_proj[k % 2], side));
  }
  for (int k = 0; k < nc; ++k) {
    SOX_CUDA_TRY(cudaStreamWaitEvent(s, ev_proj[k % 2], 0));
    SOX_TRY(tensor_steps(k, s, h->prio_high));
    SOX_CUDA_TRY(cudaEventRecord(ev_fused[k % 2], s));
    SOX_CUDA_TRY(cudaStreamWaitEvent(side, ev_fused[k % 2], 0));
    backproject(k, side);
    if (k + 2 < nc) {
      SOX_TRY(project(k + 2, side));
      SOX_CUDA_TRY(cudaEventRecord(ev_proj[k % 2], side));
    }
  }
  SOX_CUDA_TRY(cudaEventRecord(ev_join, side));
  SOX_CUDA_TRY(cudaStreamWaitEvent(s, ev_join, 0));
  SOX_CUDA_TRY(cudaGetLastError());
  return Status::ok();
}

}  // namespace sox
