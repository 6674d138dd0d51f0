// Plain CPU FP64 oracle of the FMM self-gravity solve on an octree of 8x8x8-cell
// subgrids (paper Section IV-C "Octo-Tiger"; the three-phase gravity iteration of
// Section VII-C: bottom-up, same-level cell-to-cell interactions, top-down).
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, __graft_entry__.smoke() and the
// cpu_baseline / reference leg of bench.py may load this library.  It shares no
// code, header, table or helper with the CUDA path.
//
// Everything here is written for readability, not speed: full (non-packed) Cartesian
// tensors, plain loops over every index, no blocking and no reordering beyond the
// definitions.  The scalar type is a template parameter so that the same code runs
// with std::complex<double> for complex-step derivatives.
//
// Readings of the paper that this file implements (the paper gives no formulas):
//  * Section IV-C: a leaf cell is one monopole holding the cell's mass at the cell
//    centre; interior cells carry monopole, quadrupole and octupole about their
//    centre of mass (raw, non-traceless moments).
//  * Opening criterion: cells A, B are well separated iff
//    theta * |c_A - c_B| >= (sqrt(3)/2) (h_A + h_B) with geometric cell centres c,
//    evaluated exactly in integer units (inclusive tie).
//  * Dual-tree traversal starting from all pairs of root cells: far -> M2L, both
//    leaves -> P2P, both refined on one level -> 8x8 child pairs, otherwise split
//    the refined one.
//  * M2L truncation n + k <= 3 (target order n, source order k).
//  * Angular-momentum correction (Section IV-C says the modified FMM conserves
//    angular momentum and needs the octupole): each far pair adds
//    dg_A = (m_B M3_A - m_A M3_B) : D4(X_A - X_B) / (6 m_A), dg_B = -m_A dg_A / m_B,
//    the force that the n + k <= 3 truncation drops from the (3,0) and (0,3) terms.
//  * G = 1, isolated boundaries, phi = -sum m / r.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using std::vector;
typedef std::complex<double> cplx;

inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }
inline double im(double) { return 0.0; }
inline double im(const cplx& x) { return x.imag(); }
inline double kd(int a, int b) { return a == b ? 1.0 : 0.0; }  // Kronecker delta

// ---------------------------------------------------------------------------
// Octree: every node is a leaf or has all 8 children (Section IV-C).
// ---------------------------------------------------------------------------
struct Tree {
  int n = 0, max_level = 0, n_leaf = 0, root = -1;
  vector<int> level, ijk, children, parent, octant, leaf_id;
  vector<int> leaf_nodes;
  double origin[3] = {0, 0, 0}, extent = 1;
  double h(int l) const { return extent / (8.0 * std::ldexp(1.0, l)); }
  bool is_leaf(int node) const { return children[8 * node] < 0; }
};

// Returns 0 on success, -2 for an inconsistent tree.
int build_tree(Tree& t, int n, const int32_t* level, const int32_t* ijk,
               const int32_t* children, const double* origin, double extent) {
  t.n = n;
  t.level.assign(level, level + n);
  t.ijk.assign(ijk, ijk + 3 * n);
  t.children.assign(children, children + 8 * n);
  t.parent.assign(n, -1);
  t.octant.assign(n, -1);
  t.leaf_id.assign(n, -1);
  t.leaf_nodes.clear();
  for (int d = 0; d < 3; ++d) t.origin[d] = origin[d];
  t.extent = extent;
  t.root = -1;
  t.max_level = 0;
  for (int i = 0; i < n; ++i) {
    if (level[i] < 0 || level[i] > 14) return -2;
    if (level[i] == 0) {
      if (t.root >= 0) return -2;
      t.root = i;
    }
    t.max_level = std::max(t.max_level, level[i]);
    int nc = 0;
    for (int o = 0; o < 8; ++o) nc += children[8 * i + o] >= 0;
    if (nc != 0 && nc != 8) return -2;
    for (int o = 0; o < 8; ++o) {
      int c = children[8 * i + o];
      if (c < 0) continue;
      if (c >= n || t.parent[c] >= 0 || level[c] != level[i] + 1) return -2;
      int ox = o & 1, oy = (o >> 1) & 1, oz = (o >> 2) & 1;
      if (ijk[3 * c] != 2 * ijk[3 * i] + ox || ijk[3 * c + 1] != 2 * ijk[3 * i + 1] + oy ||
          ijk[3 * c + 2] != 2 * ijk[3 * i + 2] + oz)
        return -2;
      t.parent[c] = i;
      t.octant[c] = o;
    }
  }
  if (t.root < 0) return -2;
  for (int i = 0; i < n; ++i)
    if (i != t.root && t.parent[i] < 0) return -2;
  for (int i = 0; i < n; ++i)
    if (t.is_leaf(i)) {
      t.leaf_id[i] = t.n_leaf++;
      t.leaf_nodes.push_back(i);
    }
  return 0;
}

// A cell is (node, local) with local = a + 8 b + 64 c, a,b,c in [0,8).
inline int64_t cell_id(int node, int a, int b, int c) { return (int64_t)node * 512 + a + 8 * b + 64 * c; }
inline int cnode(int64_t id) { return (int)(id / 512); }
inline void cloc(int64_t id, int loc[3]) {
  int l = (int)(id % 512);
  loc[0] = l & 7;
  loc[1] = (l >> 3) & 7;
  loc[2] = l >> 6;
}

// Integer index of a cell within its level: I = 8 * ijk + (a, b, c).
inline void global_index(const Tree& t, int64_t id, int64_t I[3]) {
  int loc[3];
  cloc(id, loc);
  int nd = cnode(id);
  for (int d = 0; d < 3; ++d) I[d] = 8 * (int64_t)t.ijk[3 * nd + d] + loc[d];
}

// Geometric centre: origin + h_l (I + 1/2).
inline void centre(const Tree& t, int64_t id, double x[3]) {
  int64_t I[3];
  global_index(t, id, I);
  double h = t.h(t.level[cnode(id)]);
  for (int d = 0; d < 3; ++d) x[d] = t.origin[d] + h * ((double)I[d] + 0.5);
}

// Children of an interior cell: cells 2I + e (e in {0,1}^3) of the next level,
// which live in child node octant (a>>2, b>>2, c>>2) at local 2(a&3)+e.
inline void child_cells(const Tree& t, int64_t id, int64_t out[8]) {
  int loc[3];
  cloc(id, loc);
  int nd = cnode(id);
  int o = (loc[0] >> 2) + 2 * (loc[1] >> 2) + 4 * (loc[2] >> 2);
  int ch = t.children[8 * nd + o];
  int k = 0;
  for (int ez = 0; ez < 2; ++ez)
    for (int ey = 0; ey < 2; ++ey)
      for (int ex = 0; ex < 2; ++ex)
        out[k++] = cell_id(ch, 2 * (loc[0] & 3) + ex, 2 * (loc[1] & 3) + ey, 2 * (loc[2] & 3) + ez);
}

inline int64_t parent_cell(const Tree& t, int64_t id) {
  int nd = cnode(id);
  int p = t.parent[nd];
  if (p < 0) return -1;
  int o = t.octant[nd];
  int loc[3];
  cloc(id, loc);
  return cell_id(p, 4 * (o & 1) + (loc[0] >> 1), 4 * ((o >> 1) & 1) + (loc[1] >> 1), 4 * ((o >> 2) & 1) + (loc[2] >> 1));
}

// Opening criterion, exact: with coordinates in units of h_f / 2 (f = finer level)
// the centres are integers C = (2I + 1) 2^(f - l), and
// theta |c_A - c_B| >= (sqrt 3 / 2)(h_A + h_B)  <=>  theta^2 Q >= 3 S^2
// with Q = |C_A - C_B|^2 and S = 2^(f - l_A) + 2^(f - l_B).
inline bool well_separated(const Tree& t, int64_t A, int64_t B, double theta) {
  int la = t.level[cnode(A)], lb = t.level[cnode(B)];
  int lf = std::max(la, lb);
  int64_t IA[3], IB[3];
  global_index(t, A, IA);
  global_index(t, B, IB);
  int64_t Q = 0;
  for (int d = 0; d < 3; ++d) {
    int64_t ca = (2 * IA[d] + 1) << (lf - la);
    int64_t cb = (2 * IB[d] + 1) << (lf - lb);
    Q += (ca - cb) * (ca - cb);
  }
  int64_t S = ((int64_t)1 << (lf - la)) + ((int64_t)1 << (lf - lb));
  return theta * theta * (double)Q >= 3.0 * (double)(S * S);
}

// ---------------------------------------------------------------------------
// Dual-tree traversal (reading of Section VII-C's "same-level cell-to-cell
// interactions on each tree level").  The visitor receives every unordered pair
// once with kind 0 (far: M2L) or 1 (both leaves, not far: P2P).  `need` prunes the
// walk to pairs with at least one member in the needed set (empty = everything).
// ---------------------------------------------------------------------------
template <class V>
struct Walker {
  const Tree& t;
  double theta;
  const vector<char>* need;  // indexed by cell id; null = all
  V& visit;
  bool needed(int64_t c) const { return !need || (*need)[c]; }
  void pair(int64_t A, int64_t B) {
    if (!needed(A) && !needed(B)) return;
    if (well_separated(t, A, B, theta)) {
      visit(A, B, 0);
      return;
    }
    bool la = t.is_leaf(cnode(A)), lb = t.is_leaf(cnode(B));
    if (la && lb) {
      visit(A, B, 1);
      return;
    }
    int lvA = t.level[cnode(A)], lvB = t.level[cnode(B)];
    int64_t ca[8], cb[8];
    if (!la && !lb && lvA == lvB) {
      child_cells(t, A, ca);
      child_cells(t, B, cb);
      for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) pair(ca[i], cb[j]);
    } else if (!la && (lb || lvA < lvB)) {
      child_cells(t, A, ca);
      for (int i = 0; i < 8; ++i) pair(ca[i], B);
    } else {
      child_cells(t, B, cb);
      for (int j = 0; j < 8; ++j) pair(A, cb[j]);
    }
  }
  void self(int64_t C) {
    if (!needed(C) || t.is_leaf(cnode(C))) return;
    int64_t c[8];
    child_cells(t, C, c);
    for (int i = 0; i < 8; ++i)
      for (int j = i + 1; j < 8; ++j) pair(c[i], c[j]);
    for (int i = 0; i < 8; ++i) self(c[i]);
  }
  void run() {
    vector<int64_t> roots;
    for (int l = 0; l < 512; ++l) roots.push_back((int64_t)t.root * 512 + l);
    for (size_t i = 0; i < roots.size(); ++i)
      for (size_t j = i + 1; j < roots.size(); ++j) pair(roots[i], roots[j]);
    for (size_t i = 0; i < roots.size(); ++i) self(roots[i]);
  }
};

// ---------------------------------------------------------------------------
// Cartesian derivative tensors D^(n) = grad^n (1/|R|), n = 0..4, full storage.
// ---------------------------------------------------------------------------
template <typename T>
struct DT {
  T D0, D1[3], D2[3][3], D3[3][3][3], D4[3][3][3][3];
};

template <typename T>
void derivative_tensors(const T R[3], DT<T>& d) {
  T r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
  T r = std::sqrt(r2);
  T i1 = 1.0 / r;
  T i3 = i1 / r2, i5 = i3 / r2, i7 = i5 / r2, i9 = i7 / r2;
  d.D0 = i1;
  for (int a = 0; a < 3; ++a) d.D1[a] = -R[a] * i3;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) d.D2[a][b] = 3.0 * R[a] * R[b] * i5 - kd(a, b) * i3;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        d.D3[a][b][c] = -15.0 * R[a] * R[b] * R[c] * i7 +
                        3.0 * (kd(a, b) * R[c] + kd(a, c) * R[b] + kd(b, c) * R[a]) * i5;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        for (int e = 0; e < 3; ++e)
          d.D4[a][b][c][e] =
              105.0 * R[a] * R[b] * R[c] * R[e] * i9 -
              15.0 *
                  (kd(a, b) * R[c] * R[e] + kd(a, c) * R[b] * R[e] + kd(a, e) * R[b] * R[c] +
                   kd(b, c) * R[a] * R[e] + kd(b, e) * R[a] * R[c] + kd(c, e) * R[a] * R[b]) *
                  i7 +
              3.0 * (kd(a, b) * kd(c, e) + kd(a, c) * kd(b, e) + kd(a, e) * kd(b, c)) * i5;
}

// Multipole of a cell about its expansion centre X (the centre of mass):
// m, raw quadrupole M2_ab = sum m s_a s_b, raw octupole M3_abc = sum m s_a s_b s_c.
template <typename T>
struct Mp {
  T m;
  T X[3];
  T M2[3][3];
  T M3[3][3][3];
};

// Local (Taylor) expansion: L^(n) = n-th derivative of phi at the cell's centre,
// plus the uniform angular-momentum correction dg carried down unshifted.
template <typename T>
struct Loc {
  T L0, L1[3], L2[3][3], L3[3][3][3], dg[3];
};

template <typename T>
void zero(Mp<T>& p) {
  p.m = 0.0;
  for (int a = 0; a < 3; ++a) {
    p.X[a] = 0.0;
    for (int b = 0; b < 3; ++b) {
      p.M2[a][b] = 0.0;
      for (int c = 0; c < 3; ++c) p.M3[a][b][c] = 0.0;
    }
  }
}
template <typename T>
void zero(Loc<T>& L) {
  L.L0 = 0.0;
  for (int a = 0; a < 3; ++a) {
    L.L1[a] = 0.0;
    L.dg[a] = 0.0;
    for (int b = 0; b < 3; ++b) {
      L.L2[a][b] = 0.0;
      for (int c = 0; c < 3; ++c) L.L3[a][b][c] = 0.0;
    }
  }
}

// M2M (parallel-axis rule, Section IV-C "moments computed about the centers of
// mass"): parent from its 8 children, each given about its own centre of mass.
template <typename T>
void m2m(const Mp<T>* ch, int nch, Mp<T>& P) {
  zero(P);
  for (int i = 0; i < nch; ++i) P.m += ch[i].m;
  for (int a = 0; a < 3; ++a) {
    T s = 0.0;
    for (int i = 0; i < nch; ++i) s += ch[i].m * ch[i].X[a];
    P.X[a] = s / P.m;
  }
  for (int i = 0; i < nch; ++i) {
    const Mp<T>& c = ch[i];
    T d[3];
    for (int a = 0; a < 3; ++a) d[a] = c.X[a] - P.X[a];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        P.M2[a][b] += c.M2[a][b] + c.m * d[a] * d[b];
        for (int e = 0; e < 3; ++e)
          P.M3[a][b][e] += c.M3[a][b][e] + c.M2[a][b] * d[e] + c.M2[a][e] * d[b] + c.M2[b][e] * d[a] +
                           c.m * d[a] * d[b] * d[e];
      }
  }
}

// M2L of source B into target A, R = X_A - X_B:
//   L_A^(n) += - sum_{k <= 3 - n} ((-1)^k / k!) M_B^(k) :k D^(n+k)(R),  M^(1) = 0,
// plus the angular-momentum correction dg_A (see file header).
template <typename T>
void m2l(const Mp<T>& A, const Mp<T>& B, Loc<T>& L, bool correction) {
  T R[3];
  for (int a = 0; a < 3; ++a) R[a] = A.X[a] - B.X[a];
  DT<T> D;
  derivative_tensors(R, D);
  // n = 0: k = 0, 2, 3
  T q2 = 0.0, q3 = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      q2 += B.M2[a][b] * D.D2[a][b];
      for (int c = 0; c < 3; ++c) q3 += B.M3[a][b][c] * D.D3[a][b][c];
    }
  L.L0 += -(B.m * D.D0 + 0.5 * q2 - q3 / 6.0);
  // n = 1: k = 0, 2
  for (int a = 0; a < 3; ++a) {
    T s = 0.0;
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) s += B.M2[b][c] * D.D3[a][b][c];
    L.L1[a] += -(B.m * D.D1[a] + 0.5 * s);
  }
  // n = 2, 3: k = 0
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      L.L2[a][b] += -(B.m * D.D2[a][b]);
      for (int c = 0; c < 3; ++c) L.L3[a][b][c] += -(B.m * D.D3[a][b][c]);
    }
  if (correction) {
    for (int a = 0; a < 3; ++a) {
      T s = 0.0;
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c)
          for (int e = 0; e < 3; ++e) s += (B.m * A.M3[b][c][e] - A.m * B.M3[b][c][e]) * D.D4[a][b][c][e];
      L.dg[a] += s / (6.0 * A.m);
    }
  }
}

// Taylor shift of a cubic local expansion from the parent centre to the child
// centre, delta = X_child - X_parent, added into the child's own expansion.
template <typename T>
void l2l(const Loc<T>& P, const T delta[3], Loc<T>& C) {
  const T* d = delta;
  T t0 = P.L0;
  for (int a = 0; a < 3; ++a) {
    t0 += P.L1[a] * d[a];
    for (int b = 0; b < 3; ++b) {
      t0 += 0.5 * P.L2[a][b] * d[a] * d[b];
      for (int c = 0; c < 3; ++c) t0 += P.L3[a][b][c] * d[a] * d[b] * d[c] / 6.0;
    }
  }
  C.L0 += t0;
  for (int a = 0; a < 3; ++a) {
    T t1 = P.L1[a];
    for (int b = 0; b < 3; ++b) {
      t1 += P.L2[a][b] * d[b];
      for (int c = 0; c < 3; ++c) t1 += 0.5 * P.L3[a][b][c] * d[b] * d[c];
    }
    C.L1[a] += t1;
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      T t2 = P.L2[a][b];
      for (int c = 0; c < 3; ++c) t2 += P.L3[a][b][c] * d[c];
      C.L2[a][b] += t2;
      for (int c = 0; c < 3; ++c) C.L3[a][b][c] += P.L3[a][b][c];
    }
  for (int a = 0; a < 3; ++a) C.dg[a] += P.dg[a];
}

// ---------------------------------------------------------------------------
// The solve.
// ---------------------------------------------------------------------------
template <typename T>
struct Solver {
  const Tree& t;
  double theta;
  bool correction;
  vector<Mp<T>> mp;  // all cells, id = node * 512 + local

  Solver(const Tree& tr, double th, bool corr) : t(tr), theta(th), correction(corr) {}

  // P2M at leaf cells (m = rho h^3 at the cell centre), then M2M bottom-up.
  void upward(const T* rho) {
    mp.assign((size_t)t.n * 512, Mp<T>());
    for (int nd = 0; nd < t.n; ++nd)
      for (int l = 0; l < 512; ++l) zero(mp[(size_t)nd * 512 + l]);
    for (int nd = 0; nd < t.n; ++nd) {
      if (!t.is_leaf(nd)) continue;
      double h = t.h(t.level[nd]);
      for (int l = 0; l < 512; ++l) {
        int64_t id = (int64_t)nd * 512 + l;
        Mp<T>& p = mp[id];
        p.m = rho[(size_t)t.leaf_id[nd] * 512 + l] * (h * h * h);
        double x[3];
        centre(t, id, x);
        for (int a = 0; a < 3; ++a) p.X[a] = x[a];
      }
    }
    for (int lv = t.max_level - 1; lv >= 0; --lv) {
#pragma omp parallel for schedule(dynamic, 1)
      for (int nd = 0; nd < t.n; ++nd) {
        if (t.level[nd] != lv || t.is_leaf(nd)) continue;
        for (int l = 0; l < 512; ++l) {
          int64_t id = (int64_t)nd * 512 + l, ch[8];
          child_cells(t, id, ch);
          Mp<T> c[8];
          for (int i = 0; i < 8; ++i) c[i] = mp[ch[i]];
          m2m(c, 8, mp[id]);
        }
      }
    }
  }

  // Interactions and downward pass for the cells in `need` (ancestor-closed);
  // fills L (indexed like mp) and the direct P2P sums for needed leaf cells.
  int64_t work = 0;  // ordered interactions evaluated by the last interact_down

  void interact_down(const vector<char>& need, vector<Loc<T>>& L, vector<T>& pphi, vector<T>& pg) {
    struct Pr {
      int64_t tgt, src;
      int kind;
    };
    vector<Pr> prs;
    auto visit = [&](int64_t A, int64_t B, int kind) {
      if (need[A]) prs.push_back({A, B, kind});
      if (need[B]) prs.push_back({B, A, kind});
    };
    Walker<decltype(visit)> w{t, theta, &need, visit};
    w.run();
    std::stable_sort(prs.begin(), prs.end(), [](const Pr& a, const Pr& b) { return a.tgt < b.tgt; });
    vector<size_t> start;
    vector<int64_t> tg;
    for (size_t i = 0; i < prs.size(); ++i)
      if (i == 0 || prs[i].tgt != prs[i - 1].tgt) {
        start.push_back(i);
        tg.push_back(prs[i].tgt);
      }
    start.push_back(prs.size());
    work = (int64_t)prs.size();
    L.assign(mp.size(), Loc<T>());
    pphi.assign(mp.size(), T(0.0));
    pg.assign(3 * mp.size(), T(0.0));
    for (size_t i = 0; i < L.size(); ++i) zero(L[i]);
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < (long)tg.size(); ++k) {
      int64_t A = tg[k];
      for (size_t i = start[k]; i < start[k + 1]; ++i) {
        const Mp<T>& src = mp[prs[i].src];
        if (prs[i].kind == 0) {
          m2l(mp[A], src, L[A], correction);
        } else {  // P2P between two leaf cells: exact point masses
          T R[3];
          for (int a = 0; a < 3; ++a) R[a] = mp[A].X[a] - src.X[a];
          T r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
          T r = std::sqrt(r2);
          pphi[A] += -src.m / r;
          for (int a = 0; a < 3; ++a) pg[3 * A + a] += -src.m * R[a] / (r2 * r);
        }
      }
    }
    // top-down Taylor shifts, level by level
    for (int lv = 1; lv <= t.max_level; ++lv) {
#pragma omp parallel for schedule(dynamic, 1)
      for (int nd = 0; nd < t.n; ++nd) {
        if (t.level[nd] != lv) continue;
        for (int l = 0; l < 512; ++l) {
          int64_t id = (int64_t)nd * 512 + l;
          if (!need[id]) continue;
          int64_t p = parent_cell(t, id);
          T d[3];
          for (int a = 0; a < 3; ++a) d[a] = mp[id].X[a] - mp[p].X[a];
          l2l(L[p], d, L[id]);
        }
      }
    }
  }
};

// needed set: requested leaf cells and all their ancestors
vector<char> needed_cells(const Tree& t, const uint8_t* leaf_mask) {
  vector<char> need((size_t)t.n * 512, 0);
  for (int nd = 0; nd < t.n; ++nd) {
    if (!t.is_leaf(nd)) continue;
    for (int l = 0; l < 512; ++l) {
      size_t k = (size_t)t.leaf_id[nd] * 512 + l;
      if (leaf_mask && !leaf_mask[k]) continue;
      int64_t c = (int64_t)nd * 512 + l;
      while (c >= 0 && !need[c]) {
        need[c] = 1;
        c = parent_cell(t, c);
      }
    }
  }
  return need;
}

// Leaf-cell outputs: phi = L0 + P2P, g = -L1 + dg + P2P (SoA g: [3][n_leaf*512]).
template <typename T, typename F>
void leaf_outputs(const Tree& t, const vector<char>& need, const vector<Loc<T>>& L, const vector<T>& pphi,
                  const vector<T>& pg, F store) {
  size_t nl = (size_t)t.n_leaf * 512;
  for (int nd = 0; nd < t.n; ++nd) {
    if (!t.is_leaf(nd)) continue;
    for (int l = 0; l < 512; ++l) {
      int64_t id = (int64_t)nd * 512 + l;
      size_t k = (size_t)t.leaf_id[nd] * 512 + l;
      if (!need[id]) continue;
      T phi = L[id].L0 + pphi[id];
      T g[3];
      for (int a = 0; a < 3; ++a) g[a] = -L[id].L1[a] + L[id].dg[a] + pg[3 * id + a];
      store(k, nl, phi, g);
    }
  }
}

// ---------------------------------------------------------------------------
// Vector-Jacobian product (reverse of every step above, float64, full tensors).
// ---------------------------------------------------------------------------

// D^(5) = grad^5 (1/|R|) from the expansion of derivatives of a radial function:
// for the multi-index with exponents (a, b, c),
//   d^a_x d^b_y d^c_z F(r) = sum_{i,j,k} H(a,i) H(b,j) H(c,k) x^(a-2i) y^(b-2j) z^(c-2k) F_{n-i-j-k},
//   H(a,i) = a! / (2^i i! (a-2i)!),  F_m = (r^-1 d/dr)^m (1/r) = (-1)^m (2m-1)!! r^-(2m+1).
double hermite_coef(int a, int i) {
  double f = 1;
  for (int k = 2; k <= a; ++k) f *= k;
  double d = std::ldexp(1.0, i);
  for (int k = 2; k <= i; ++k) d *= k;
  for (int k = 2; k <= a - 2 * i; ++k) d *= k;
  return f / d;
}

void derivative5(const double R[3], double D5[3][3][3][3][3]) {
  double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
  double F[6];
  F[0] = 1.0 / std::sqrt(r2);
  for (int m = 1; m < 6; ++m) F[m] = -(2.0 * m - 1.0) * F[m - 1] / r2;
  double pw[3][6];
  for (int d = 0; d < 3; ++d) {
    pw[d][0] = 1.0;
    for (int k = 1; k < 6; ++k) pw[d][k] = pw[d][k - 1] * R[d];
  }
  double byexp[6][6];  // [a][b], c = 5 - a - b
  for (int a = 0; a <= 5; ++a)
    for (int b = 0; a + b <= 5; ++b) {
      int c = 5 - a - b;
      double s = 0;
      for (int i = 0; 2 * i <= a; ++i)
        for (int j = 0; 2 * j <= b; ++j)
          for (int k = 0; 2 * k <= c; ++k)
            s += hermite_coef(a, i) * hermite_coef(b, j) * hermite_coef(c, k) * pw[0][a - 2 * i] * pw[1][b - 2 * j] *
                 pw[2][c - 2 * k] * F[5 - i - j - k];
      byexp[a][b] = s;
    }
  for (int i0 = 0; i0 < 3; ++i0)
    for (int i1 = 0; i1 < 3; ++i1)
      for (int i2 = 0; i2 < 3; ++i2)
        for (int i3 = 0; i3 < 3; ++i3)
          for (int i4 = 0; i4 < 3; ++i4) {
            int e[3] = {0, 0, 0};
            e[i0]++, e[i1]++, e[i2]++, e[i3]++, e[i4]++;
            D5[i0][i1][i2][i3][i4] = byexp[e[0]][e[1]];
          }
}

// Adjoint of the M2L of B into A (see m2l): given Lb = dS/dL_A (and dS/d dg_A in
// Lb.dg), adds dS/d(multipole of A) into Ab and dS/d(multipole of B) into Bb.
void m2l_vjp(const Mp<double>& A, const Mp<double>& B, const Loc<double>& Lb, bool correction, Mp<double>& Ab,
             Mp<double>& Bb) {
  double R[3];
  for (int a = 0; a < 3; ++a) R[a] = A.X[a] - B.X[a];
  DT<double> D;
  derivative_tensors(R, D);
  static thread_local double D5[3][3][3][3][3];
  derivative5(R, D5);
  // adjoints of the derivative tensors
  double D0b = -B.m * Lb.L0, D1b[3], D2b[3][3], D3b[3][3][3], D4b[3][3][3][3];
  for (int a = 0; a < 3; ++a) {
    D1b[a] = -B.m * Lb.L1[a];
    for (int b = 0; b < 3; ++b) {
      D2b[a][b] = -0.5 * Lb.L0 * B.M2[a][b] - B.m * Lb.L2[a][b];
      for (int c = 0; c < 3; ++c) {
        D3b[a][b][c] = Lb.L0 * B.M3[a][b][c] / 6.0 - 0.5 * Lb.L1[a] * B.M2[b][c] - B.m * Lb.L3[a][b][c];
        for (int e = 0; e < 3; ++e)
          D4b[a][b][c][e] = correction ? Lb.dg[a] * (B.m * A.M3[b][c][e] - A.m * B.M3[b][c][e]) / (6.0 * A.m) : 0.0;
      }
    }
  }
  // multipole adjoints
  double mB = -Lb.L0 * D.D0;
  for (int a = 0; a < 3; ++a) {
    mB -= Lb.L1[a] * D.D1[a];
    for (int b = 0; b < 3; ++b) {
      mB -= Lb.L2[a][b] * D.D2[a][b];
      for (int c = 0; c < 3; ++c) mB -= Lb.L3[a][b][c] * D.D3[a][b][c];
    }
  }
  for (int b = 0; b < 3; ++b)
    for (int c = 0; c < 3; ++c) {
      double s = Lb.L0 * D.D2[b][c];
      for (int a = 0; a < 3; ++a) s += Lb.L1[a] * D.D3[a][b][c];
      Bb.M2[b][c] += -0.5 * s;
    }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) Bb.M3[a][b][c] += Lb.L0 * D.D3[a][b][c] / 6.0;
  if (correction) {
    double mA = 0;
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        for (int e = 0; e < 3; ++e) {
          double t = 0;  // sum_a dg_a D4_abce
          for (int a = 0; a < 3; ++a) t += Lb.dg[a] * D.D4[a][b][c][e];
          mB += t * A.M3[b][c][e] / (6.0 * A.m);
          Bb.M3[b][c][e] += -t / 6.0;
          Ab.M3[b][c][e] += B.m * t / (6.0 * A.m);
          mA += -B.m * t * A.M3[b][c][e] / (6.0 * A.m * A.m);
        }
    Ab.m += mA;
  }
  Bb.m += mB;
  // position adjoints through R = X_A - X_B
  for (int f = 0; f < 3; ++f) {
    double s = D0b * D.D1[f];
    for (int a = 0; a < 3; ++a) {
      s += D1b[a] * D.D2[a][f];
      for (int b = 0; b < 3; ++b) {
        s += D2b[a][b] * D.D3[a][b][f];
        for (int c = 0; c < 3; ++c) {
          s += D3b[a][b][c] * D.D4[a][b][c][f];
          for (int e = 0; e < 3; ++e) s += D4b[a][b][c][e] * D5[a][b][c][e][f];
        }
      }
    }
    Ab.X[f] += s;
    Bb.X[f] -= s;
  }
}

// Adjoint of the P2P of leaf cell B into leaf cell A (positions are fixed).
void p2p_vjp(const Mp<double>& A, const Mp<double>& B, double phib, const double* gb, Mp<double>& Bb) {
  double R[3];
  for (int a = 0; a < 3; ++a) R[a] = A.X[a] - B.X[a];
  double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
  double r = std::sqrt(r2);
  double s = -phib / r;
  for (int a = 0; a < 3; ++a) s += -gb[a] * R[a] / (r2 * r);
  Bb.m += s;
}

// Adjoint of the Taylor shift (l2l): given Cb = dS/dC (C the child's expansion),
// adds into Pb = dS/dP and returns dS/d delta in db.
void l2l_vjp(const Loc<double>& P, const double d[3], const Loc<double>& Cb, Loc<double>& Pb, double db[3]) {
  Pb.L0 += Cb.L0;
  for (int a = 0; a < 3; ++a) {
    Pb.L1[a] += Cb.L0 * d[a] + Cb.L1[a];
    Pb.dg[a] += Cb.dg[a];
    for (int b = 0; b < 3; ++b) {
      Pb.L2[a][b] += 0.5 * Cb.L0 * d[a] * d[b] + Cb.L1[a] * d[b] + Cb.L2[a][b];
      for (int c = 0; c < 3; ++c)
        Pb.L3[a][b][c] += Cb.L0 * d[a] * d[b] * d[c] / 6.0 + 0.5 * Cb.L1[a] * d[b] * d[c] + Cb.L2[a][b] * d[c] +
                          Cb.L3[a][b][c];
    }
  }
  // S = Cb . shift(P, d); differentiate every d factor
  for (int f = 0; f < 3; ++f) {
    double s = 0;
    // from L0' = L0 + L1.d + L2:dd/2 + L3:ddd/6
    s += Cb.L0 * P.L1[f];
    for (int a = 0; a < 3; ++a) {
      s += Cb.L0 * 0.5 * (P.L2[f][a] + P.L2[a][f]) * d[a];
      for (int b = 0; b < 3; ++b)
        s += Cb.L0 * (P.L3[f][a][b] + P.L3[a][f][b] + P.L3[a][b][f]) * d[a] * d[b] / 6.0;
    }
    // from L1'_a = L1_a + L2_ab d_b + L3_abc d_b d_c / 2
    for (int a = 0; a < 3; ++a) {
      s += Cb.L1[a] * P.L2[a][f];
      for (int b = 0; b < 3; ++b) s += Cb.L1[a] * 0.5 * (P.L3[a][f][b] + P.L3[a][b][f]) * d[b];
    }
    // from L2'_ab = L2_ab + L3_abc d_c
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) s += Cb.L2[a][b] * P.L3[a][b][f];
    db[f] = s;
  }
}

// Adjoint of m2m: given Pb = dS/dP, adds dS/d(child) into chb[i].
void m2m_vjp(const Mp<double>* ch, int nch, const Mp<double>& P, const Mp<double>& Pb, Mp<double>* chb) {
  double Xb[3] = {Pb.X[0], Pb.X[1], Pb.X[2]};  // grows with the d_c = X_c - X_P terms
  for (int i = 0; i < nch; ++i) {
    const Mp<double>& c = ch[i];
    double d[3], db[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) d[a] = c.X[a] - P.X[a];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        // M2_P,ab += M2_c,ab + m d_a d_b
        chb[i].M2[a][b] += Pb.M2[a][b];
        chb[i].m += Pb.M2[a][b] * d[a] * d[b];
        db[a] += Pb.M2[a][b] * c.m * d[b];
        db[b] += Pb.M2[a][b] * c.m * d[a];
        for (int e = 0; e < 3; ++e) {
          // M3_P,abe += M3_c + M2_ab d_e + M2_ae d_b + M2_be d_a + m d_a d_b d_e
          double w = Pb.M3[a][b][e];
          chb[i].M3[a][b][e] += w;
          chb[i].M2[a][b] += w * d[e];
          chb[i].M2[a][e] += w * d[b];
          chb[i].M2[b][e] += w * d[a];
          chb[i].m += w * d[a] * d[b] * d[e];
          db[e] += w * (c.M2[a][b] + c.m * d[a] * d[b]);
          db[b] += w * (c.M2[a][e] + c.m * d[a] * d[e]);
          db[a] += w * (c.M2[b][e] + c.m * d[b] * d[e]);
        }
      }
    for (int a = 0; a < 3; ++a) {
      chb[i].X[a] += db[a];
      Xb[a] -= db[a];
    }
  }
  // X_P = sum m_c X_c / m_P and m_P = sum m_c
  for (int i = 0; i < nch; ++i) {
    for (int a = 0; a < 3; ++a) {
      chb[i].X[a] += Xb[a] * ch[i].m / P.m;
      chb[i].m += Xb[a] * (ch[i].X[a] - P.X[a]) / P.m;
    }
    chb[i].m += Pb.m;
  }
}

// Packed orders shared by the exported arrays (documented in oracle/__init__.py):
// multipole: m, X0..2, M2 {00,01,02,11,12,22}, M3 {000,001,002,011,012,022,111,112,122,222}
// local:     L0, L1 0..2, L2 {..6}, L3 {..10}, dg 0..2
const int P2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
const int P3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                       {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};

}  // namespace

extern "C" {

// Bottom-up pass only.  mp_out: [20][n_nodes*512] packed multipoles, every node.
int oracle_upward(int n, const int32_t* level, const int32_t* ijk, const int32_t* children, const double* origin,
                  double extent, const double* rho, double* mp_out) {
  Tree t;
  int rc = build_tree(t, n, level, ijk, children, origin, extent);
  if (rc) return rc;
  Solver<double> s(t, 0.5, true);
  s.upward(rho);
  size_t nc = (size_t)n * 512;
  for (size_t i = 0; i < nc; ++i) {
    const Mp<double>& p = s.mp[i];
    mp_out[0 * nc + i] = p.m;
    for (int a = 0; a < 3; ++a) mp_out[(1 + a) * nc + i] = p.X[a];
    for (int q = 0; q < 6; ++q) mp_out[(4 + q) * nc + i] = p.M2[P2[q][0]][P2[q][1]];
    for (int q = 0; q < 10; ++q) mp_out[(10 + q) * nc + i] = p.M3[P3[q][0]][P3[q][1]][P3[q][2]];
  }
  return 0;
}

// Full FMM.  leaf_mask (n_leaf*512 bytes, may be null = all) selects the leaf cells
// whose phi/g are computed; others are left untouched.  flags bit0: apply the
// angular-momentum correction.  loc_out (may be null): [23][n_nodes*512] final local
// expansions (after the downward pass) of needed cells, NaN elsewhere.  work_out
// (may be null): number of ordered interactions (M2L + P2P) evaluated.
int oracle_fmm(int n, const int32_t* level, const int32_t* ijk, const int32_t* children, const double* origin,
               double extent, const double* rho, double theta, int flags, const uint8_t* leaf_mask, double* phi,
               double* g, double* loc_out, int64_t* work_out) {
  Tree t;
  int rc = build_tree(t, n, level, ijk, children, origin, extent);
  if (rc) return rc;
  Solver<double> s(t, theta, flags & 1);
  s.upward(rho);
  vector<char> need = needed_cells(t, leaf_mask);
  vector<Loc<double>> L;
  vector<double> pphi, pg;
  s.interact_down(need, L, pphi, pg);
  if (work_out) *work_out = s.work;
  leaf_outputs(t, need, L, pphi, pg, [&](size_t k, size_t nl, double ph, const double* gg) {
    phi[k] = ph;
    for (int a = 0; a < 3; ++a) g[a * nl + k] = gg[a];
  });
  if (loc_out) {
    size_t nc = (size_t)n * 512;
    for (size_t i = 0; i < nc; ++i) {
      const Loc<double>& l = L[i];
      double v[23];
      v[0] = l.L0;
      for (int a = 0; a < 3; ++a) v[1 + a] = l.L1[a];
      for (int q = 0; q < 6; ++q) v[4 + q] = l.L2[P2[q][0]][P2[q][1]];
      for (int q = 0; q < 10; ++q) v[10 + q] = l.L3[P3[q][0]][P3[q][1]][P3[q][2]];
      for (int a = 0; a < 3; ++a) v[20 + a] = l.dg[a];
      for (int f = 0; f < 23; ++f) loc_out[f * nc + i] = need[i] ? v[f] : NAN;
    }
  }
  return 0;
}

// Complex-step directional derivative: runs the same FMM with rho + i*eps*u and
// returns Im(phi)/eps, Im(g)/eps for the selected leaf cells (and Re parts).
int oracle_fmm_jvp(int n, const int32_t* level, const int32_t* ijk, const int32_t* children, const double* origin,
                   double extent, const double* rho, const double* u, double eps, double theta, int flags,
                   const uint8_t* leaf_mask, double* phi, double* g, double* dphi, double* dg) {
  Tree t;
  int rc = build_tree(t, n, level, ijk, children, origin, extent);
  if (rc) return rc;
  size_t nl = (size_t)t.n_leaf * 512;
  vector<cplx> rc_in(nl);
  for (size_t i = 0; i < nl; ++i) rc_in[i] = cplx(rho[i], eps * u[i]);
  Solver<cplx> s(t, theta, flags & 1);
  s.upward(rc_in.data());
  vector<char> need = needed_cells(t, leaf_mask);
  vector<Loc<cplx>> L;
  vector<cplx> pphi, pg;
  s.interact_down(need, L, pphi, pg);
  leaf_outputs(t, need, L, pphi, pg, [&](size_t k, size_t nl2, cplx ph, const cplx* gg) {
    phi[k] = ph.real();
    dphi[k] = ph.imag() / eps;
    for (int a = 0; a < 3; ++a) {
      g[a * nl2 + k] = gg[a].real();
      dg[a * nl2 + k] = gg[a].imag() / eps;
    }
  });
  return 0;
}

// Direct N^2 sum over all leaf cells (point masses at cell centres), for the
// selected targets: phi_i = -sum_j m_j / r_ij, g_i = -sum_j m_j (x_i - x_j) / r_ij^3.
int oracle_direct(int n, const int32_t* level, const int32_t* ijk, const int32_t* children, const double* origin,
                  double extent, const double* rho, const uint8_t* leaf_mask, double* phi, double* g) {
  Tree t;
  int rc = build_tree(t, n, level, ijk, children, origin, extent);
  if (rc) return rc;
  size_t nl = (size_t)t.n_leaf * 512;
  vector<double> x(3 * nl), m(nl);
  for (int nd = 0; nd < t.n; ++nd) {
    if (!t.is_leaf(nd)) continue;
    double h = t.h(t.level[nd]);
    for (int l = 0; l < 512; ++l) {
      size_t k = (size_t)t.leaf_id[nd] * 512 + l;
      centre(t, (int64_t)nd * 512 + l, &x[3 * k]);
      m[k] = rho[k] * (h * h * h);
    }
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (long i = 0; i < (long)nl; ++i) {
    if (leaf_mask && !leaf_mask[i]) continue;
    double p = 0, gg[3] = {0, 0, 0};
    for (size_t j = 0; j < nl; ++j) {
      if ((size_t)i == j) continue;
      double R[3];
      for (int a = 0; a < 3; ++a) R[a] = x[3 * i + a] - x[3 * j + a];
      double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
      double r = std::sqrt(r2);
      p += -m[j] / r;
      for (int a = 0; a < 3; ++a) gg[a] += -m[j] * R[a] / (r2 * r);
    }
    phi[i] = p;
    for (int a = 0; a < 3; ++a) g[a * nl + i] = gg[a];
  }
  return 0;
}

// Ordered interaction counts from a full walk:
// out[0] same-level M2L, out[1] cross-level M2L, out[2] same-level P2P, out[3] cross-level P2P.
int oracle_counts(int n, const int32_t* level, const int32_t* ijk, const int32_t* children, const double* origin,
                  double extent, double theta, int64_t* out) {
  Tree t;
  int rc = build_tree(t, n, level, ijk, children, origin, extent);
  if (rc) return rc;
  int64_t c[4] = {0, 0, 0, 0};
  auto visit = [&](int64_t A, int64_t B, int kind) {
    bool same = t.level[cnode(A)] == t.level[cnode(B)];
    c[2 * kind + (same ? 0 : 1)] += 2;
  };
  Walker<decltype(visit)> w{t, theta, nullptr, visit};
  w.run();
  for (int i = 0; i < 4; ++i) out[i] = c[i];
  return 0;
}

// Pair coverage: for every ordered pair of distinct leaf cells (i, j), the number of
// interactions (far pairs of their ancestors-or-self, or P2P) that account for it.
// Writes a n_leafcells x n_leafcells int32 matrix; for tests on tiny trees only.
int oracle_coverage(int n, const int32_t* level, const int32_t* ijk, const int32_t* children, const double* origin,
                    double extent, double theta, int32_t* cover) {
  Tree t;
  int rc = build_tree(t, n, level, ijk, children, origin, extent);
  if (rc) return rc;
  size_t nl = (size_t)t.n_leaf * 512;
  std::memset(cover, 0, sizeof(int32_t) * nl * nl);
  // leaf descendants of every cell
  auto leaves_under = [&](int64_t c, vector<size_t>& out) {
    vector<int64_t> st{c};
    while (!st.empty()) {
      int64_t x = st.back();
      st.pop_back();
      int nd = cnode(x);
      if (t.is_leaf(nd)) {
        out.push_back((size_t)t.leaf_id[nd] * 512 + (size_t)(x % 512));
      } else {
        int64_t ch[8];
        child_cells(t, x, ch);
        for (int i = 0; i < 8; ++i) st.push_back(ch[i]);
      }
    }
  };
  auto visit = [&](int64_t A, int64_t B, int) {
    vector<size_t> la, lb;
    leaves_under(A, la);
    leaves_under(B, lb);
    for (size_t i : la)
      for (size_t j : lb) {
        cover[i * nl + j] += 1;
        cover[j * nl + i] += 1;
      }
  };
  Walker<decltype(visit)> w{t, theta, nullptr, visit};
  w.run();
  return 0;
}

// Unit-level entry points for the pins.
void oracle_dtensors(const double* R, double* out /* 1+3+9+27+81 */) {
  DT<double> d;
  derivative_tensors(R, d);
  int k = 0;
  out[k++] = d.D0;
  for (int a = 0; a < 3; ++a) out[k++] = d.D1[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) out[k++] = d.D2[a][b];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) out[k++] = d.D3[a][b][c];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        for (int e = 0; e < 3; ++e) out[k++] = d.D4[a][b][c][e];
}

static void unpack_mp(const double* v, Mp<double>& p) {
  p.m = v[0];
  for (int a = 0; a < 3; ++a) p.X[a] = v[1 + a];
  for (int q = 0; q < 6; ++q) {
    int a = P2[q][0], b = P2[q][1];
    p.M2[a][b] = p.M2[b][a] = v[4 + q];
  }
  for (int q = 0; q < 10; ++q) {
    int a = P3[q][0], b = P3[q][1], c = P3[q][2];
    p.M3[a][b][c] = p.M3[a][c][b] = p.M3[b][a][c] = p.M3[b][c][a] = p.M3[c][a][b] = p.M3[c][b][a] = v[10 + q];
  }
}
static void pack_loc(const Loc<double>& l, double* v) {
  v[0] = l.L0;
  for (int a = 0; a < 3; ++a) v[1 + a] = l.L1[a];
  for (int q = 0; q < 6; ++q) v[4 + q] = l.L2[P2[q][0]][P2[q][1]];
  for (int q = 0; q < 10; ++q) v[10 + q] = l.L3[P3[q][0]][P3[q][1]][P3[q][2]];
  for (int a = 0; a < 3; ++a) v[20 + a] = l.dg[a];
}
static void unpack_loc(const double* v, Loc<double>& l) {
  l.L0 = v[0];
  for (int a = 0; a < 3; ++a) l.L1[a] = v[1 + a];
  for (int q = 0; q < 6; ++q) {
    int a = P2[q][0], b = P2[q][1];
    l.L2[a][b] = l.L2[b][a] = v[4 + q];
  }
  for (int q = 0; q < 10; ++q) {
    int a = P3[q][0], b = P3[q][1], c = P3[q][2];
    l.L3[a][b][c] = l.L3[a][c][b] = l.L3[b][a][c] = l.L3[b][c][a] = l.L3[c][a][b] = l.L3[c][b][a] = v[10 + q];
  }
  for (int a = 0; a < 3; ++a) l.dg[a] = v[20 + a];
}

// One M2L of packed source B into packed target A (20 values each); out: 23 values.
void oracle_m2l_pair(const double* A, const double* B, int correction, double* out) {
  Mp<double> a, b;
  unpack_mp(A, a);
  unpack_mp(B, b);
  Loc<double> L;
  zero(L);
  m2l(a, b, L, correction != 0);
  pack_loc(L, out);
}

// M2M of nch packed children (20 values each, contiguous) into one packed parent.
void oracle_m2m(const double* ch, int nch, double* out) {
  vector<Mp<double>> c(nch);
  for (int i = 0; i < nch; ++i) unpack_mp(ch + 20 * i, c[i]);
  Mp<double> P;
  m2m(c.data(), nch, P);
  out[0] = P.m;
  for (int a = 0; a < 3; ++a) out[1 + a] = P.X[a];
  for (int q = 0; q < 6; ++q) out[4 + q] = P.M2[P2[q][0]][P2[q][1]];
  for (int q = 0; q < 10; ++q) out[10 + q] = P.M3[P3[q][0]][P3[q][1]][P3[q][2]];
}

// L2L of a packed parent expansion (23 values) by delta into zero; out: 23 values.
void oracle_l2l(const double* parent, const double* delta, double* out) {
  Loc<double> P, C;
  unpack_loc(parent, P);
  zero(C);
  l2l(P, delta, C);
  pack_loc(C, out);
}

// Thread count of the OpenMP loops (timing of the oracle at 1 thread and at all
// cores); returns the count now in effect.  No effect on any result: every loop
// writes disjoint outputs.
int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

}  // extern "C"

namespace {

// drho = J^T (dphi, dg) of the full solve, by the reverse of each step:
// L2P^T seeds, L2L^T (finest to coarsest), M2L^T / P2P^T over every ordered pair,
// M2M^T (coarsest to finest), P2M^T.
int fmm_vjp(const Tree& t, const double* rho, double theta, bool corr, const double* phib, const double* gb,
            double* rhob) {
  Solver<double> s(t, theta, corr);
  s.upward(rho);
  const size_t NC = s.mp.size();
  vector<char> all(NC, 1);
  vector<Loc<double>> L;
  vector<double> pphi, pg;
  s.interact_down(all, L, pphi, pg);  // final local expansions of every cell
  struct Pr {
    int64_t tgt, src;
    int kind;
  };
  vector<Pr> prs;
  auto visit = [&](int64_t A, int64_t B, int kind) {
    prs.push_back({A, B, kind});
    prs.push_back({B, A, kind});
  };
  Walker<decltype(visit)> w{t, theta, nullptr, visit};
  w.run();
  // seeds at leaf cells: phi = L0 + P2P, g = -L1 + dg + P2P
  vector<Loc<double>> Lb(NC);
  for (auto& x : Lb) zero(x);
  vector<double> pphib(NC, 0.0), pgb(3 * NC, 0.0);
  const size_t nl = (size_t)t.n_leaf * 512;
  for (int nd = 0; nd < t.n; ++nd) {
    if (!t.is_leaf(nd)) continue;
    for (int l = 0; l < 512; ++l) {
      size_t id = (size_t)nd * 512 + l, k = (size_t)t.leaf_id[nd] * 512 + l;
      Lb[id].L0 = phib[k];
      pphib[id] = phib[k];
      for (int a = 0; a < 3; ++a) {
        Lb[id].L1[a] = -gb[a * nl + k];
        Lb[id].dg[a] = gb[a * nl + k];
        pgb[3 * id + a] = gb[a * nl + k];
      }
    }
  }
  vector<Mp<double>> mpb(NC);
  for (auto& x : mpb) zero(x);
  // L2L^T
  for (int lv = t.max_level; lv >= 1; --lv)
    for (int nd = 0; nd < t.n; ++nd) {
      if (t.level[nd] != lv) continue;
      for (int l = 0; l < 512; ++l) {
        int64_t c = (int64_t)nd * 512 + l, p = parent_cell(t, c);
        double d[3], db[3];
        for (int a = 0; a < 3; ++a) d[a] = s.mp[c].X[a] - s.mp[p].X[a];
        l2l_vjp(L[p], d, Lb[c], Lb[p], db);
        for (int a = 0; a < 3; ++a) {
          mpb[c].X[a] += db[a];
          mpb[p].X[a] -= db[a];
        }
      }
    }
  // M2L^T and P2P^T: target-side gradients grouped by target, source-side by source
  for (int side = 0; side < 2; ++side) {
    std::stable_sort(prs.begin(), prs.end(), [&](const Pr& a, const Pr& b) {
      return side == 0 ? a.tgt < b.tgt : a.src < b.src;
    });
    vector<size_t> start;
    for (size_t i = 0; i < prs.size(); ++i)
      if (i == 0 || (side == 0 ? prs[i].tgt != prs[i - 1].tgt : prs[i].src != prs[i - 1].src)) start.push_back(i);
    start.push_back(prs.size());
    const long ngroups = (long)start.size() - 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (long g = 0; g < ngroups; ++g) {
      for (size_t i = start[g]; i < start[g + 1]; ++i) {
        const Pr& pr = prs[i];
        Mp<double> Ab, Bb;
        zero(Ab);
        zero(Bb);
        if (pr.kind == 0)
          m2l_vjp(s.mp[pr.tgt], s.mp[pr.src], Lb[pr.tgt], corr, Ab, Bb);
        else if (side == 1)
          p2p_vjp(s.mp[pr.tgt], s.mp[pr.src], pphib[pr.tgt], &pgb[3 * pr.tgt], Bb);
        Mp<double>& dst = side == 0 ? mpb[pr.tgt] : mpb[pr.src];
        const Mp<double>& v = side == 0 ? Ab : Bb;
        dst.m += v.m;
        for (int a = 0; a < 3; ++a) {
          dst.X[a] += v.X[a];
          for (int b = 0; b < 3; ++b) {
            dst.M2[a][b] += v.M2[a][b];
            for (int c = 0; c < 3; ++c) dst.M3[a][b][c] += v.M3[a][b][c];
          }
        }
      }
    }
  }
  // M2M^T, coarsest to finest
  for (int lv = 0; lv < t.max_level; ++lv)
    for (int nd = 0; nd < t.n; ++nd) {
      if (t.level[nd] != lv || t.is_leaf(nd)) continue;
      for (int l = 0; l < 512; ++l) {
        int64_t id = (int64_t)nd * 512 + l, ch[8];
        child_cells(t, id, ch);
        Mp<double> c[8], cb[8];
        for (int i = 0; i < 8; ++i) {
          c[i] = s.mp[ch[i]];
          zero(cb[i]);
        }
        m2m_vjp(c, 8, s.mp[id], mpb[id], cb);
        for (int i = 0; i < 8; ++i) {
          Mp<double>& dst = mpb[ch[i]];
          dst.m += cb[i].m;
          for (int a = 0; a < 3; ++a) {
            dst.X[a] += cb[i].X[a];
            for (int b = 0; b < 3; ++b) {
              dst.M2[a][b] += cb[i].M2[a][b];
              for (int e = 0; e < 3; ++e) dst.M3[a][b][e] += cb[i].M3[a][b][e];
            }
          }
        }
      }
    }
  // P2M^T: m = rho h^3 (leaf positions and zero higher moments are constants)
  for (int nd = 0; nd < t.n; ++nd) {
    if (!t.is_leaf(nd)) continue;
    double h = t.h(t.level[nd]);
    for (int l = 0; l < 512; ++l)
      rhob[(size_t)t.leaf_id[nd] * 512 + l] = mpb[(size_t)nd * 512 + l].m * (h * h * h);
  }
  return 0;
}

}  // namespace

extern "C" {

// Vector-Jacobian product of the full solve: drho = (dphi/drho)^T phib + (dg/drho)^T gb.
int oracle_fmm_vjp(int n, const int32_t* level, const int32_t* ijk, const int32_t* children, const double* origin,
                   double extent, const double* rho, double theta, int flags, const double* phib, const double* gb,
                   double* rhob) {
  Tree t;
  int rc = build_tree(t, n, level, ijk, children, origin, extent);
  if (rc) return rc;
  return fmm_vjp(t, rho, theta, flags & 1, phib, gb, rhob);
}

// D^(5) (243 values, row-major) for the pins.
void oracle_dtensor5(const double* R, double* out) {
  double D5[3][3][3][3][3];
  derivative5(R, D5);
  std::memcpy(out, D5, sizeof(D5));
}

}  // extern "C"
