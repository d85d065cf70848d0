// The closed-shell (S)CCSD functions as a tensor-operation graph.
#pragma once

#include "graph.h"

namespace sccsd {

struct EnergyResidual {
  int E0 = -1, O1 = -1, O2 = -1;
  // dressed one-body intermediates whose diagonals approximate the diagonal of
  // the Jacobian (the Davidson preconditioner): Fvv'[b][c], Foo'[k][j]
  int Fvvi = -1, Fooi = -1;
  int Govov = -1;  // g_iajb as [i][j][a][b] (undressed)
};

// Builds E0 = <HF|Hbar|HF> and Omega_mu = <mu~|Hbar|HF> (Sec. 2.1) in the
// T1-transformed form Hbar = exp(-T2) Hhat exp(T2), Hhat = exp(-T1) H exp(T1)
// (Sec. 2.4.2). Inputs: t1 [v][o] ("ai"), t2 [o][o][v][v] ("ijab", full and
// symmetric), L [J][n][n], h [n][n], delta [o][o] (identity).
EnergyResidual build_energy_residual(Graph& g, int t1, int t2, int L, int h, int delta);

// <mu~|Hhat R1(x1) R2(y2)|HF> (the building block of zeta <mu~|[Hhat, X3]|HF>,
// Sec. 2.4.2) from mixed derivatives of the CCSD functions at T2 = 0.
struct Xi {
  int X1 = -1, X2 = -1;
};
// er0 must be build_energy_residual(g, t1, t2zero, ...) whose ops are primal0;
// t2zero is an input that always holds zeros.
Xi build_xi(Graph& g, int t1, int t2zero, const EnergyResidual& er0,
            const Graph::Ranges& primal0, int x1, int y2);

}  // namespace sccsd
