// Library-internal hooks shared by the translation units of libozdmrg (not part of the C ABI).
#pragma once
#include <string>
#include <vector>

#include "ozdmrg.h"

namespace oz {

// Records `msg` as the calling thread's oz_last_error() text and returns `code`.
int api_fail(int code, const std::string& msg);

// Device ordinal of a context.
int ctx_device(const oz_ctx* c);

// Read-only views of an H_eff handle.
long long heff_dim(const oz_heff* h);
int heff_device(const oz_heff* h);
int heff_nsm(const oz_heff* h);
oz_ctx* heff_ctx(const oz_heff* h);
// Device vector (length heff_dim) of the diagonal of H_eff, built by oz_heff_create.
const double* heff_diag_ptr(const oz_heff* h);

// Builds the diagonal of H_eff = sum over tasks of coef L (x) R into d_diag (length psioff[nsec]):
// only tasks with src == dst contribute, diag[(q,i,j)] = sum_t L_t[i][i] (coef_t R_t[j][j]).
// Synchronous (called while the caller's operator blocks are alive).
int build_heff_diag(int nsec, const int* m, const int* n, const long long* psioff, int ntask, const oz_task* tasks,
                    double* d_diag);

// A batch of independent emulated products C = op(A) op(B), all sliced in one pass and multiplied
// in one grouped launch (S digits stored, level s used).  op(A) = A (M x K, row-major, lda) or,
// with transA, the transpose of a row-major K x M matrix (lda = its row stride); op(B) = B (K x N
// row-major, ldb) or, with transB, the transpose of a row-major N x K matrix; C: M x N row-major
// (ldc), overwritten.  Synchronous; uses the context's workspace.
struct EmuJob {
  const double* A;
  long long lda;
  int transA;
  const double* B;
  long long ldb;
  int transB;  // op(B) = the transpose of a row-major N x K matrix (ldb = its row stride)
  double* C;
  long long ldc;
  int M, N, K;
};
int emulated_batch(oz_ctx* c, const std::vector<EmuJob>& jobs, int S, int s, cudaStream_t st);

// Exponent-gap histograms of the operator blocks of a new emulated handle (oz_select.cu).
int heff_operator_hist(oz_heff* h, const oz_task* tasks);

}  // namespace oz
