// The C problem statement of include/mgiga.h into the host representation.
#pragma once

#include "../../include/mgiga.h"
#include "host.hpp"

namespace mgiga {
// validates *P (throws SetupError(MGIGA_EINVAL, ...) with the reason) and fills pr
void import_problem(const mgiga_problem* P, Problem& pr);
// lv levels: the finest on the problem's knots, each coarser one on every other
// breakpoint (Sec. 2, nested spaces); layouts, numbering and shared copies
void init_levels(const Problem& pr, int lv, std::vector<Level>& L);
// the finest operator by quadrature (Sec. 2-3), Dirichlet DoFs eliminated
void assemble_finest(const Problem& pr, std::vector<Level>& L);
// the coarser operators A_{l-1} = P_l^T A_l P_l (Eq. a:galerkin) and the
// transfers P_l (T[l], l >= 1; knot insertion, Sec. 4)
void galerkin_hierarchy(std::vector<Level>& L, std::vector<Transfer>& T);
}  // namespace mgiga
