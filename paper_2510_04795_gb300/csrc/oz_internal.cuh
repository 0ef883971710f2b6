// Library-internal hooks shared by the translation units of libozdmrg (not part of the C ABI).
#pragma once
#include <string>

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

// Exponent-gap histograms of the operator blocks of a new emulated handle (oz_select.cu).
int heff_operator_hist(oz_heff* h, const oz_task* tasks);

}  // namespace oz
