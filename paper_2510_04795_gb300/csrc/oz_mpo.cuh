// Matrix product operator of the ab initio Hamiltonian (host side).
//
//   H = sum_{pq,s} h_pq a+_{ps} a_{qs} + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}
//
// on L spatial orbitals (one MPO site per orbital, local basis |0>, |up>, |down>, |up down>),
// Jordan-Wigner order orbital-major with up before down.  Every term is reordered so that its
// operators stand in ascending site order (the sign of the permutation goes into its coefficient);
// the local operator of a term on site j is then (product of its operators on j) P^(number of its
// operators right of j), P = (-1)^n the site parity.  The automaton that sums the terms keys the
// state of a term at bond b (between site b and b+1) by its operators left of the bond when fewer
// (or, at a tie, when the left part of the chain is not longer) than right of it, and by its
// operators right of the bond otherwise; a term's coefficient is applied on the one site where
// it switches from the left key to the right key.  Left-keyed states are normal operators of the
// left block, right-keyed ones are complementary operators (sums over integrals) on the left: the
// bond dimension grows as O(L^2).  The environments of a two-site DMRG bond indexed by these states
// give the effective Hamiltonian as sum_w L_w (x) R_w.
#pragma once
#include <string>
#include <vector>

namespace oz {

struct QN {
  int n;  // electrons
  int s;  // 2 Sz
};

struct MpoEntry {
  int row, col;   // state at the bond left of the site, state at the bond right of it
  double m[16];   // local operator, m[s_out * 4 + s_in]
};

struct Mpo {
  int L = 0;
  // states of bond b = -1..L-1 at index b + 1: change of (n, 2Sz) that the left part applies
  std::vector<std::vector<QN>> delta;
  std::vector<std::vector<MpoEntry>> W;  // W[j]: entries of site j
  int chi(int b) const { return (int)delta[b + 1].size(); }
};

// Quantum numbers of the site states 0..3.
constexpr int SITE_N[4] = {0, 1, 1, 2};
constexpr int SITE_S[4] = {0, 1, -1, 0};

// h1: L x L, eri: L^4 chemist (pq|rs) at ((p L + q) L + r) L + s, both host FP64.
int build_mpo(const double* h1, const double* eri, int L, Mpo* out, std::string* err);

}  // namespace oz
