// MPO of the ab initio Hamiltonian (host code; see oz_mpo.cuh) and its verification entries.
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ozdmrg.h"
#include "oz_internal.cuh"
#include "oz_mpo.cuh"

namespace oz {
namespace {

struct Op {
  int x;    // spin orbital 2p + sigma
  int dag;  // 1 = creation
};

struct Term {
  double c;
  int m;
  Op op[4];
};

using Mat4 = std::array<double, 16>;

Mat4 local_matrix(int x, int dag) {
  Mat4 a{};
  const int up = (x & 1) == 0;
  // creation operators; annihilation is the transpose (real matrices)
  if (up) {
    a[1 * 4 + 0] = 1.0;   // |up>      <- |0>
    a[3 * 4 + 2] = 1.0;   // |up down> <- |down>
  } else {
    a[2 * 4 + 0] = 1.0;   // |down>    <- |0>
    a[3 * 4 + 1] = -1.0;  // |up down> <- |up>   (a+_down passes a+_up)
  }
  if (!dag) {
    Mat4 t{};
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) t[i * 4 + j] = a[j * 4 + i];
    return t;
  }
  return a;
}

Mat4 matmul4(const Mat4& a, const Mat4& b) {
  Mat4 c{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += a[i * 4 + k] * b[k * 4 + j];
      c[i * 4 + j] = s;
    }
  return c;
}

Mat4 identity4() {
  Mat4 a{};
  for (int i = 0; i < 4; ++i) a[i * 4 + i] = 1.0;
  return a;
}

Mat4 parity4() {
  Mat4 a{};
  a[0] = 1.0;
  a[5] = -1.0;
  a[10] = -1.0;
  a[15] = 1.0;
  return a;
}

// Stable reorder by site; returns the sign of the permutation (operators on different sites
// anticommute; those on one site keep their order).
double sort_by_site(Term& t) {
  double sign = 1.0;
  for (int i = 1; i < t.m; ++i)
    for (int k = i; k > 0 && (t.op[k - 1].x >> 1) > (t.op[k].x >> 1); --k) {
      std::swap(t.op[k - 1], t.op[k]);
      sign = -sign;
    }
  return sign;
}

}  // namespace

int build_mpo(const double* h1, const double* eri, int L, Mpo* out, std::string* err) {
  if (L < 2 || L > 64) {
    *err = "L must be in 2..64";
    return OZ_EINVAL;
  }
  // ---- terms
  std::vector<Term> terms;
  for (int p = 0; p < L; ++p)
    for (int q = 0; q < L; ++q)
      for (int sg = 0; sg < 2; ++sg) {
        double c = h1[p * L + q];
        if (c == 0.0) continue;
        Term t{c, 2, {{2 * p + sg, 1}, {2 * q + sg, 0}, {0, 0}, {0, 0}}};
        terms.push_back(t);
      }
  for (int p = 0; p < L; ++p)
    for (int q = 0; q < L; ++q)
      for (int r = 0; r < L; ++r)
        for (int s = 0; s < L; ++s) {
          const double v = eri[((size_t)(p * L + q) * L + r) * L + s];
          if (v == 0.0) continue;
          for (int sg = 0; sg < 2; ++sg)
            for (int tg = 0; tg < 2; ++tg) {
              const int a = 2 * p + sg, b = 2 * r + tg, cc = 2 * s + tg, d = 2 * q + sg;
              if (a == b || cc == d) continue;  // a+_x a+_x = a_x a_x = 0
              Term t{0.5 * v, 4, {{a, 1}, {b, 1}, {cc, 0}, {d, 0}}};
              terms.push_back(t);
            }
        }
  for (auto& t : terms) t.c *= sort_by_site(t);

  // ---- bond states
  Mpo& M = *out;
  M = Mpo();
  M.L = L;
  M.delta.assign(L + 1, {});
  M.W.assign(L, {});
  std::vector<std::map<std::vector<int>, int>> keys(L + 1);
  auto key_of = [&](const Term& t, int b, int* tag) {
    int nl = 0;
    while (nl < t.m && (t.op[nl].x >> 1) <= b) ++nl;
    const int nr = t.m - nl;
    bool left;
    if (nl == 0) left = true;
    else if (nr == 0) left = false;
    else if (nl != nr) left = nl < nr;
    else left = (b + 1) <= (L - b - 1);
    std::vector<int> k;
    k.push_back(left ? 0 : 1);
    if (left)
      for (int i = 0; i < nl; ++i) k.push_back(t.op[i].x * 2 + t.op[i].dag);
    else
      for (int i = nl; i < t.m; ++i) k.push_back(t.op[i].x * 2 + t.op[i].dag);
    *tag = left ? 0 : 1;
    return k;
  };
  auto qn_of_key = [](const std::vector<int>& k) {
    QN d{0, 0};
    for (size_t i = 1; i < k.size(); ++i) {
      const int x = k[i] >> 1, dag = k[i] & 1, up = (x & 1) == 0;
      const int sgn = dag ? 1 : -1;
      d.n += sgn;
      d.s += sgn * (up ? 1 : -1);
    }
    if (k[0] == 1) {  // right-keyed: the left part applies the opposite change
      d.n = -d.n;
      d.s = -d.s;
    }
    return d;
  };
  auto state = [&](int b, const std::vector<int>& k) {
    auto& mp = keys[b + 1];
    auto it = mp.find(k);
    if (it != mp.end()) return it->second;
    const int id = (int)M.delta[b + 1].size();
    mp.emplace(k, id);
    M.delta[b + 1].push_back(qn_of_key(k));
    return id;
  };
  // fixed ids: bond -1 holds only the empty left key, bond L-1 only the empty right key; the
  // inner bonds start with both
  state(-1, {0});
  for (int b = 0; b < L - 1; ++b) {
    state(b, {0});
    state(b, {1});
  }
  state(L - 1, {1});

  // ---- transitions
  std::vector<std::map<std::pair<int, int>, Mat4>> setm(L), addm(L);
  const Mat4 P = parity4();
  for (const Term& t : terms) {
    int tag_prev;
    std::vector<int> kprev = key_of(t, -1, &tag_prev);
    int sprev = state(-1, kprev);
    for (int j = 0; j < L; ++j) {
      int tag;
      std::vector<int> k = key_of(t, j, &tag);
      const int s = state(j, k);
      Mat4 loc = identity4();
      int nright = 0;
      for (int i = 0; i < t.m; ++i) {
        const int site = t.op[i].x >> 1;
        if (site == j) loc = matmul4(loc, local_matrix(t.op[i].x, t.op[i].dag));
        else if (site > j) ++nright;
      }
      if (nright & 1) loc = matmul4(loc, P);
      const auto rc = std::make_pair(sprev, s);
      if (tag_prev == tag) {
        auto it = setm[j].find(rc);
        if (it == setm[j].end()) {
          setm[j].emplace(rc, loc);
        } else {
          for (int e = 0; e < 16; ++e)
            if (it->second[e] != loc[e]) {
              *err = "inconsistent MPO transition";
              return OZ_EINVAL;
            }
        }
      } else if (tag_prev == 0 && tag == 1) {
        auto& a = addm[j][rc];
        for (int e = 0; e < 16; ++e) a[e] += t.c * loc[e];
      } else {
        *err = "MPO term switches from a right key back to a left key";
        return OZ_EINVAL;
      }
      sprev = s;
      tag_prev = tag;
    }
  }
  // identity transitions of the empty keys on every site (needed even where no term passes)
  for (int j = 0; j < L; ++j) {
    if (j < L - 1) setm[j].emplace(std::make_pair(0, 0), identity4());  // I_L -> I_L
    if (j > 0) {
      const int rprev = 1;  // I_R at bond j-1 (index 1 on inner bonds)
      const int rnext = (j == L - 1) ? 0 : 1;
      setm[j].emplace(std::make_pair(rprev, rnext), identity4());  // I_R -> I_R
    }
  }
  for (int j = 0; j < L; ++j) {
    for (auto& kv : setm[j]) {
      MpoEntry e;
      e.row = kv.first.first;
      e.col = kv.first.second;
      std::memcpy(e.m, kv.second.data(), sizeof(e.m));
      M.W[j].push_back(e);
    }
    for (auto& kv : addm[j]) {
      bool nz = false;
      for (double v : kv.second) nz = nz || v != 0.0;
      if (!nz) continue;
      MpoEntry e;
      e.row = kv.first.first;
      e.col = kv.first.second;
      std::memcpy(e.m, kv.second.data(), sizeof(e.m));
      M.W[j].push_back(e);
    }
  }
  return OZ_OK;
}

}  // namespace oz

extern "C" int oz_mpo_bond_dims(const double* h1, const double* eri, int L, int* chi) {
  if (!h1 || !eri || !chi) return oz::api_fail(OZ_EINVAL, "null argument");
  oz::Mpo M;
  std::string err;
  if (int rc = oz::build_mpo(h1, eri, L, &M, &err)) return oz::api_fail(rc, err);
  for (int b = -1; b < L; ++b) chi[b + 1] = M.chi(b);
  return OZ_OK;
}

extern "C" int oz_mpo_dense(const double* h1, const double* eri, int L, double* out) {
  if (!h1 || !eri || !out) return oz::api_fail(OZ_EINVAL, "null argument");
  if (L < 2 || L > 4) return oz::api_fail(OZ_EINVAL, "oz_mpo_dense supports L in 2..4");
  oz::Mpo M;
  std::string err;
  if (int rc = oz::build_mpo(h1, eri, L, &M, &err)) return oz::api_fail(rc, err);
  // T[w]: operator on sites 0..j for bond-j state w, index sum_i s_i 4^i (site 0 least significant)
  std::vector<std::vector<double>> T(1, std::vector<double>(1, 1.0));
  int dim = 1;
  for (int j = 0; j < L; ++j) {
    const int nd = dim * 4;
    std::vector<std::vector<double>> Tn(M.chi(j), std::vector<double>((size_t)nd * nd, 0.0));
    for (const auto& e : M.W[j]) {
      const auto& A = T[e.row];
      auto& B = Tn[e.col];
      for (int so = 0; so < 4; ++so)
        for (int si = 0; si < 4; ++si) {
          const double w = e.m[so * 4 + si];
          if (w == 0.0) continue;
          for (int r = 0; r < dim; ++r)
            for (int c = 0; c < dim; ++c) {
              const double a = A[(size_t)r * dim + c];
              if (a != 0.0) B[(size_t)(so * dim + r) * nd + (si * dim + c)] += w * a;
            }
        }
    }
    T.swap(Tn);
    dim = nd;
  }
  std::memcpy(out, T[0].data(), sizeof(double) * (size_t)dim * dim);
  return OZ_OK;
}
