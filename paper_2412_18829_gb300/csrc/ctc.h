// Complex split-precision GEMMs on the tensor cores and the momentum-resolved SOX
// chain on them (ctc.cu).
#pragma once
#include <cuda_fp16.h>

#include "internal.h"

namespace sox {

// A split operand: `batch` blocks of `rows` real rows, each Kp2 = 64*ceil(2K/64) FP16
// values (hi and lo), and one FP32 factor per real row that undoes its scale.
struct CSplit {
  __half *hi = nullptr, *lo = nullptr;
  float *unscale = nullptr;
  int batch = 0, rows = 0, Kp2 = 0;
  long long bstride = 0;   // rows between consecutive batches (0: `rows`)
  // rows [r0, r0 + rows) of every batch of this split, as an operand of its own
  CSplit view(long long r0, int nrows) const {
    CSplit v = *this;
    const long long off = r0 * Kp2;
    v.hi = hi + off;
    v.lo = lo + off;
    v.unscale = unscale + r0;
    v.bstride = bstride ? bstride : rows;
    v.rows = nrows;
    return v;
  }
};
int csplit_kp2(int K);
size_t csplit_bytes(int batch, int rows_real, int K);
CSplit csplit_take(Arena &ar, int batch, int rows_real, int K);

// Complex rows of a strided source (element (b, r, k) at src + b*sb + (r/R2)*sr1 +
// (r%R2)*sr2 + k*sk complex elements; R2 <= 0 means row r at r*sr1), FP64 or FP32.
//   csplit_a: `rows` complex rows -> `rows` real rows (the A operand).
//   csplit_b: `cols` complex rows -> 2*cols real rows (the B operand), with the
//             conjugations of the product folded in.
void csplit_a(const void *src, bool f32, long long sb, long long sr1, long long sr2, int R2, long long sk, int batch,
              int rows, int K, const CSplit &out, cudaStream_t s);
void csplit_b(const void *src, bool f32, long long sb, long long sr1, long long sr2, int R2, long long sk, int batch,
              int cols, int K, bool conjA, bool conjB, const CSplit &out, cudaStream_t s);

// B operand of the mixed tensors from X: pair (q, k') = q*n_k + k', rows (a, b) of
// conj(X^{k'-q}[Q][a]) X^{k'}[Q][b] (2 n^2 real rows per pair), K = Q.
void csplit_pairs(const double *X, const int *sub, int nk, int N, int n, const CSplit &out, cudaStream_t s);

// C[b][i][j] = alpha sum_k opA(A[zA])[i][k] opB(B[zB])[j][k], complex FP32 interleaved, C row
// stride ldc and batch stride sCb in floats (multiples of 4, C 16-byte aligned);
// zA = idxA ? idxA[b] : (A.batch == 1 ? 0 : b), zB likewise.
Status cgemm_tc(sox_handle h, const CSplit &A, const CSplit &B, int batch, const int *idxA, const int *idxB,
                float alpha, float *C, long long ldc, long long sCb, cudaStream_t s, bool accumulate = false);

// Real operands: `rows` real rows of K values (Kp2 = 64*ceil(K/64)), element (b, r, k) at
// src + b*sb + (r/R2)*sr1 + (r%R2)*sr2 + k*sk (real elements), FP64 or FP32.  cgemm_tc
// multiplies real splits as well (C[b][i][j] = alpha sum_k A[i][k] B[j][k], FP32).
int rsplit_kp(int K);
size_t rsplit_bytes(int batch, int rows, int K);
CSplit rsplit_take(Arena &ar, int batch, int rows, int K);
// mul (optional, FP32): each element is multiplied by mul at the same offset without
// the batch term (a Hadamard factor shared by all batches)
void rsplit(const void *src, bool f32, long long sb, long long sr1, long long sr2, int R2, long long sk, int batch,
            int rows, int K, const CSplit &out, cudaStream_t s, const float *mul = nullptr);

// D[i0 + il][k][e] += sum_{q1,q2} C[(q2, k+q1), il][e] B[(q1, k+q1-q2), il][e]  for il < ct and
// e < NN; B and C FP32 complex with element (pair p, il, e) at p*sP + il*sI + e (complex
// units), D FP64 complex [.][k][NN] with stride sDi per i.
Status kpoint_D_f32(const float *B, const float *C, long long sP, long long sI, const int *add, const int *sub,
                    const int mesh[3], long long NN, int ct, int i0, long long sDi, double *D, cudaStream_t s);

// Split-precision forms of the momentum-resolved chain (handle precision SOX_PREC_F16X2).
size_t kpoint_tc_bytes(sox_handle h, const sox_problem *p, bool two);
Status kpoint_sigma_tc(sox_handle h, const sox_problem *p, const double *G, const double *X, const double *U1,
                       const double *U2, double *Sigma, Arena &ar, cudaStream_t s);
size_t kpoint_dynamic_tc_bytes(sox_handle h, const sox_problem *p, int n_omega);
Status kpoint_dynamic_tc(sox_handle h, const sox_problem *p, int n_omega, const double *G, const double *X,
                         const double *V, const double *Wd, const double *T_fwd, const double *T_inv, double *Sigma,
                         Arena &ar, cudaStream_t s);

}  // namespace sox
