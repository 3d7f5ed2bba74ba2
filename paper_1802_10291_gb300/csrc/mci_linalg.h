// Small dense linear algebra of the plan code (host only).
#pragma once
#include <complex>
#include <vector>

#include "mci.h"

namespace mci {

// Q = H^{-1} of one M x M system matrix H[j * M + k] = b_k(n_j) (Eq. (defH)), or its
// Moore-Penrose pseudo-inverse where sigma_min < rtol sigma_max (Remark (aequal0)), from a
// one-sided Jacobi SVD; Q[m * M + j].  policy is an MCI_SINGULAR_* value: ZERO leaves Q = 0
// at a singular matrix, ERROR returns MCI_ERR_SINGULAR.  *singular and *cond
// (sigma_max / sigma_min) describe H.
mci_status invert_system(int M, std::vector<std::complex<double>> H, double rtol, int policy,
                         std::complex<double>* Q, bool* singular, double* cond);

}  // namespace mci
