// Read access to a solver's orbitals and eigenvalues for the SCF module.
#pragma once

#include <cstdint>

#include "rsdft.h"

namespace rs {

struct SolverView {
    const void *psi;     // device [npts][nst], dtype
    const double *eig;   // device [nst], the last subspace diagonalisation's eigenvalues
    int nst, dtype;
    int64_t npts;
    double dV;
};
void solver_view(rs_solver *s, SolverView *v);

}  // namespace rs
