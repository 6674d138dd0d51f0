// Host-side planning: see plan.h.
//
// Interaction structure (reading of the paper's Section VII-C "same-level
// cell-to-cell interactions on each tree level"): two cells interact through
// their expansions when the opening criterion holds and their parents' does not.
// On one level this is a fixed stencil that depends only on the parity of the
// target cell's index; at refinement boundaries a leaf cell meets the children of
// a near refined cell, which gives the explicit cross-level pair lists.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <unordered_map>

namespace octo {

double cell_width(const Plan& p, int level) { return p.extent / (8.0 * std::ldexp(1.0, level)); }

namespace {

inline int floor_div2(int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }
inline int floor_div8(int v) { return v >= 0 ? v / 8 : -((-v + 7) / 8); }

// Opening criterion in exact integer form.  In units of half the finer cell width
// the geometric centres are C = (2 I + 1) * 2^(f - l); the criterion
// theta |c_A - c_B| >= (sqrt 3 / 2)(h_A + h_B) becomes theta^2 Q >= 3 S^2 with
// Q = |C_A - C_B|^2 and S = 2^(f - l_A) + 2^(f - l_B).
bool well_separated(double theta, int la, const int64_t* IA, int lb, const int64_t* IB) {
  int lf = la > lb ? la : lb;
  int64_t Q = 0;
  for (int d = 0; d < 3; ++d) {
    int64_t ca = (2 * IA[d] + 1) << (lf - la);
    int64_t cb = (2 * IB[d] + 1) << (lf - lb);
    Q += (ca - cb) * (ca - cb);
  }
  int64_t S = ((int64_t)1 << (lf - la)) + ((int64_t)1 << (lf - lb));
  return theta * theta * (double)Q >= 3.0 * (double)(S * S);
}

// Same-level special case (Q = 4 |d|^2, S = 2).
bool far_offset(double theta, int dx, int dy, int dz) {
  int64_t Q = 4 * (int64_t)(dx * dx + dy * dy + dz * dz);
  return theta * theta * (double)Q >= 3.0 * 4.0;
}

struct Key {
  int64_t v;
  bool operator==(const Key& o) const { return v == o.v; }
};
struct KeyHash {
  size_t operator()(const Key& k) const { return std::hash<int64_t>()(k.v); }
};
inline Key make_key(int l, int64_t i, int64_t j, int64_t k) {
  return Key{((int64_t)l << 56) | (i << 37) | (j << 18) | k};
}

// Splits the cross-level pair lists into the tabulated point-mass list (both cells
// leaves, one level apart) and the general remainder (layouts in plan.h).
void split_cross_pairs(Plan& P) {
  int RN = 0;
  for (int32_t e : P.st_near)
    for (int k = 0; k < 3; ++k) RN = std::max(RN, std::abs((int)(int8_t)((e >> (8 * k)) & 0xff)));
  // |v| <= 4 RN + 1 for a pair found from a near offset; rows must fit 16 bits
  const int na = 2 * RN + 1;
  const bool table_ok = 2 * (int64_t)na * na * na + 1 < 65536;
  P.xc_na = na;
  const int64_t zero_row = 2 * (int64_t)na * na * na;
  P.xc_table.assign(4 * (zero_row + 1), 0.0);
  for (int g = 0; g < 2; ++g) {
    const double s = g == 0 ? 4.0 : 2.0;
    for (int ax = 0; ax < na; ++ax)
      for (int ay = 0; ay < na; ++ay)
        for (int az = 0; az < na; ++az) {
          const double v[3] = {2.0 * ax + 1, 2.0 * ay + 1, 2.0 * az + 1};
          const double r = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
          double* row = &P.xc_table[4 * (g * (int64_t)na * na * na + (ax * na + ay) * na + az)];
          row[0] = s / r;
          for (int k = 0; k < 3; ++k) row[1 + k] = s * s * v[k] / (r * r * r);
        }
  }
  auto cell_index = [&](int64_t c, int64_t I[3]) {
    const int node = (int)(c / kCells), l = (int)(c % kCells);
    const int loc[3] = {l & 7, (l >> 3) & 7, l >> 6};
    for (int a = 0; a < 3; ++a) I[a] = 8 * (int64_t)P.ijk[3 * node + a] + loc[a];
  };
  // per target: tabulated entries, general entries (far ones first)
  std::vector<std::pair<int64_t, int64_t>> by_count;  // (count, slot)
  std::vector<int64_t> slot_target, tab_start(1, 0), tab_ent;
  P.xg_targets.clear();
  P.xg_start.assign(1, 0);
  P.xg_mid.clear();
  P.xg_sources.clear();
  const size_t nt = P.x_targets.size();
  for (size_t i = 0; i < nt; ++i) {
    const int64_t tg = P.x_targets[i];
    const int tn = (int)(tg / kCells), lt = P.level[tn];
    const bool t_leaf = P.children[8 * tn] < 0;
    int64_t It[3];
    cell_index(tg, It);
    const int64_t tab0 = (int64_t)tab_ent.size();
    const size_t g0 = P.xg_sources.size();
    int64_t gmid = -1;
    for (int64_t e = P.x_start[i]; e < P.x_start[i + 1]; ++e) {
      const int64_t src = P.x_sources[e];
      const int sn = (int)(src / kCells), ls = P.level[sn];
      bool tab = table_ok && t_leaf && P.children[8 * sn] < 0 && std::abs(ls - lt) == 1;
      int64_t row = 0, signs = 0;
      if (tab) {
        int64_t Is[3];
        cell_index(src, Is);
        // centres in units of half the finer cell width: fine 2 I + 1, coarse 4 I + 2
        for (int a = 0; a < 3 && tab; ++a) {
          const int64_t ct = ls > lt ? 4 * It[a] + 2 : 2 * It[a] + 1;
          const int64_t cs = ls > lt ? 2 * Is[a] + 1 : 4 * Is[a] + 2;
          const int64_t v = ct - cs, av = v < 0 ? -v : v;
          if ((av & 1) == 0 || av > 2 * na - 1) tab = false;
          row = row * na + (av - 1) / 2;
          if (v < 0) signs |= 1 << a;
        }
        row += (ls > lt ? 0 : 1) * (int64_t)na * na * na;
      }
      if (tab) {
        tab_ent.push_back(src << 20 | signs << 16 | row);
      } else {
        if (e >= P.x_mid[i] && gmid < 0) gmid = (int64_t)P.xg_sources.size();
        P.xg_sources.push_back(src);
      }
    }
    if ((int64_t)tab_ent.size() > tab0) {  // slot k spans tab_ent[tab_start[k], tab_start[k + 1])
      by_count.push_back({(int64_t)tab_ent.size() - tab0, (int64_t)slot_target.size()});
      slot_target.push_back(tg);
      tab_start.push_back((int64_t)tab_ent.size());
    }
    if (P.xg_sources.size() > g0) {
      P.xg_targets.push_back(tg);
      P.xg_mid.push_back(gmid < 0 ? (int64_t)P.xg_sources.size() : gmid);
      P.xg_start.push_back((int64_t)P.xg_sources.size());
    }
  }
  P.xc_pairs = (int64_t)tab_ent.size();
  // SELL-32: sort tabulated targets by decreasing count (ties in list order)
  std::stable_sort(by_count.begin(), by_count.end(),
                   [](const std::pair<int64_t, int64_t>& a, const std::pair<int64_t, int64_t>& b) {
                     return a.first > b.first;
                   });
  const int64_t nts = (int64_t)by_count.size(), n_slices = (nts + 31) / 32;
  P.xc_targets.assign(32 * n_slices, -1);
  P.xc_slice_off.assign(n_slices + 1, 0);
  for (int64_t s = 0; s < n_slices; ++s) {
    int64_t w = by_count[32 * s].first;  // widest target of the slice comes first
    w = (w + 3) / 4 * 4;
    P.xc_slice_off[s + 1] = P.xc_slice_off[s] + 32 * w;
  }
  P.xc_entries.assign(P.xc_slice_off[n_slices], (int64_t)zero_row);
  for (int64_t j = 0; j < nts; ++j) {
    const int64_t s = j / 32, lane = j % 32, slot = by_count[j].second;
    P.xc_targets[j] = slot_target[slot];
    const int64_t o = P.xc_slice_off[s] + lane;
    for (int64_t k = tab_start[slot]; k < tab_start[slot + 1]; ++k) P.xc_entries[o + 32 * (k - tab_start[slot])] = tab_ent[k];
  }
}

}  // namespace

int build_plan(const octo_tree_desc* desc, double theta, Plan& P) {
  if (!desc || !desc->level || !desc->ijk || !desc->children || desc->n_nodes <= 0) {
    P.error = "null or empty tree descriptor";
    return OCTO_EINVAL;
  }
  if (!(theta >= 0.433 && theta <= 1.0)) {
    P.error = "theta outside the supported range [0.433, 1]";
    return OCTO_EINVAL;
  }
  if (!(desc->extent > 0.0) || !std::isfinite(desc->extent)) {
    P.error = "extent must be positive and finite";
    return OCTO_EINVAL;
  }
  const int n = desc->n_nodes;
  P.theta = theta;
  P.extent = desc->extent;
  for (int d = 0; d < 3; ++d) P.origin[d] = desc->origin[d];

  // ---------------- validate ----------------
  int root = -1, maxl = 0;
  std::vector<int> par(n, -1), oct(n, -1);
  for (int i = 0; i < n; ++i) {
    int l = desc->level[i];
    if (l < 0 || l > kMaxLevel) {
      P.error = "node level out of range";
      return OCTO_ETREE;
    }
    for (int d = 0; d < 3; ++d) {
      int v = desc->ijk[3 * i + d];
      if (v < 0 || v >= (1 << l)) {
        P.error = "node ijk outside its level";
        return OCTO_ETREE;
      }
    }
    if (l == 0) {
      if (root >= 0) {
        P.error = "more than one root";
        return OCTO_ETREE;
      }
      root = i;
    }
    maxl = std::max(maxl, l);
    int nch = 0;
    for (int o = 0; o < 8; ++o) nch += desc->children[8 * i + o] >= 0 ? 1 : 0;
    if (nch != 0 && nch != 8) {
      P.error = "a node must be a leaf or have all 8 children";
      return OCTO_ETREE;
    }
    for (int o = 0; o < 8 && nch; ++o) {
      int c = desc->children[8 * i + o];
      if (c >= n || par[c] >= 0 || desc->level[c] != l + 1) {
        P.error = "bad child index or level";
        return OCTO_ETREE;
      }
      const int e[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
      for (int d = 0; d < 3; ++d)
        if (desc->ijk[3 * c + d] != 2 * desc->ijk[3 * i + d] + e[d]) {
          P.error = "child ijk does not match its octant";
          return OCTO_ETREE;
        }
      par[c] = i;
      oct[c] = o;
    }
  }
  if (root < 0) {
    P.error = "no root node";
    return OCTO_ETREE;
  }
  for (int i = 0; i < n; ++i)
    if (i != root && par[i] < 0) {
      P.error = "node not reachable from the root";
      return OCTO_ETREE;
    }

  // ---------------- device order: by level, then descriptor order ----------------
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return desc->level[a] < desc->level[b]; });
  P.n_nodes = n;
  P.max_level = maxl;
  P.desc_of_dnode.assign(order.begin(), order.end());
  P.dnode_of_desc.assign(n, -1);
  for (int k = 0; k < n; ++k) P.dnode_of_desc[order[k]] = k;
  P.level.resize(n);
  P.ijk.resize(3 * n);
  P.parent.assign(n, -1);
  P.octant.assign(n, -1);
  P.children.assign(8 * n, -1);
  P.leaf_id.assign(n, -1);
  P.level_start.assign(maxl + 2, 0);
  // leaf order = descriptor order of leaves
  std::vector<int> leaf_of_desc(n, -1);
  int nl = 0;
  for (int i = 0; i < n; ++i)
    if (desc->children[8 * i] < 0) leaf_of_desc[i] = nl++;
  P.n_leaf = nl;
  for (int k = 0; k < n; ++k) {
    int i = order[k];
    P.level[k] = desc->level[i];
    for (int d = 0; d < 3; ++d) P.ijk[3 * k + d] = desc->ijk[3 * i + d];
    P.parent[k] = par[i] >= 0 ? P.dnode_of_desc[par[i]] : -1;
    P.octant[k] = oct[i];
    for (int o = 0; o < 8; ++o) {
      int c = desc->children[8 * i + o];
      P.children[8 * k + o] = c >= 0 ? P.dnode_of_desc[c] : -1;
    }
    P.leaf_id[k] = leaf_of_desc[i];
    P.level_start[P.level[k] + 1] = k + 1;
  }
  for (int l = 1; l <= maxl + 1; ++l) P.level_start[l] = std::max(P.level_start[l], P.level_start[l - 1]);

  // ---------------- same-level neighbours ----------------
  std::unordered_map<Key, int, KeyHash> at;
  at.reserve(2 * n);
  for (int k = 0; k < n; ++k) at[make_key(P.level[k], P.ijk[3 * k], P.ijk[3 * k + 1], P.ijk[3 * k + 2])] = k;
  P.nbr.assign(27 * n, -1);
  for (int k = 0; k < n; ++k) {
    int s = 1 << P.level[k];
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          int64_t i = P.ijk[3 * k] + ox, j = P.ijk[3 * k + 1] + oy, kk = P.ijk[3 * k + 2] + oz;
          if (i < 0 || j < 0 || kk < 0 || i >= s || j >= s || kk >= s) continue;
          auto it = at.find(make_key(P.level[k], i, j, kk));
          if (it != at.end()) P.nbr[27 * k + (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)] = it->second;
        }
  }

  // ---------------- stencils ----------------
  const int RS = 9;
  P.st_parity.clear();
  std::vector<std::vector<int32_t>> per(8);
  for (int p = 0; p < 8; ++p) {
    const int pp[3] = {p & 1, (p >> 1) & 1, (p >> 2) & 1};
    for (int dz = -RS; dz <= RS; ++dz)
      for (int dy = -RS; dy <= RS; ++dy)
        for (int dx = -RS; dx <= RS; ++dx) {
          if (!far_offset(theta, dx, dy, dz)) continue;
          const int d[3] = {dx, dy, dz};
          int D[3];
          for (int a = 0; a < 3; ++a) D[a] = floor_div2(pp[a] + d[a]);
          if (far_offset(theta, D[0], D[1], D[2])) continue;
          if (std::abs(dx) > 8 || std::abs(dy) > 8 || std::abs(dz) > 8) {
            P.error = "theta too small: stencil leaves the 26 neighbouring subgrids";
            return OCTO_EINVAL;
          }
          per[p].push_back(pack_offset(dx, dy, dz));
        }
  }
  P.n_st = (int)per[0].size();
  for (int p = 0; p < 8; ++p) {
    if ((int)per[p].size() != P.n_st) {
      P.error = "parity stencils differ in size";
      return OCTO_EINVAL;
    }
    P.st_parity.insert(P.st_parity.end(), per[p].begin(), per[p].end());
  }
  // every near parent offset must have near grandparent offsets, so that the
  // parity stencil equals the set of pairs the tree walk reaches
  for (int Dz = -RS; Dz <= RS; ++Dz)
    for (int Dy = -RS; Dy <= RS; ++Dy)
      for (int Dx = -RS; Dx <= RS; ++Dx) {
        if (far_offset(theta, Dx, Dy, Dz)) continue;
        for (int q = 0; q < 8; ++q) {
          int G[3] = {floor_div2((q & 1) + Dx), floor_div2(((q >> 1) & 1) + Dy), floor_div2(((q >> 2) & 1) + Dz)};
          if (far_offset(theta, G[0], G[1], G[2])) {
            P.error = "theta not supported: near cells with far parents";
            return OCTO_EINVAL;
          }
        }
      }
  P.st_root.clear();
  P.st_near.clear();
  for (int dz = -7; dz <= 7; ++dz)
    for (int dy = -7; dy <= 7; ++dy)
      for (int dx = -7; dx <= 7; ++dx) {
        if (far_offset(theta, dx, dy, dz))
          P.st_root.push_back(pack_offset(dx, dy, dz));
        else if (dx || dy || dz)
          P.st_near.push_back(pack_offset(dx, dy, dz));
      }
  {  // near offsets as (d, -d) pairs: the near item sums a pair's two masses for the
     // potential and differences them for the field (kernel rows of -d are those of
     // d with the gradient part negated).  The set is symmetric and was generated in
     // lexicographic order, so entry k and entry n - 1 - k are negatives.
    const std::vector<int32_t> lex = P.st_near;
    const size_t nn = lex.size();
    P.st_near.clear();
    for (size_t k = 0; k < nn / 2; ++k) {
      P.st_near.push_back(lex[k]);
      P.st_near.push_back(lex[nn - 1 - k]);
    }
    bool paired = nn % 2 == 0;
    for (size_t k = 0; paired && k < nn; k += 2)
      for (int b = 0; b < 3; ++b)
        paired = paired && (int8_t)((P.st_near[k] >> (8 * b)) & 0xff) == -(int8_t)((P.st_near[k + 1] >> (8 * b)) & 0xff);
    if (!paired) {
      P.error = "near offsets are not symmetric";
      return OCTO_EINVAL;
    }
  }
  // per-cell entry lists by neighbour slot
  P.cell_ent.clear();
  P.cell_ent_off.assign(1, 0);
  std::vector<int32_t> cell_cnt(kCells * 27, 0);
  for (int l = 0; l < kCells; ++l) {
    const int loc[3] = {l & 7, (l >> 3) & 7, l >> 6};
    const int p = (loc[0] & 1) + 2 * (loc[1] & 1) + 4 * (loc[2] & 1);
    for (int o = 0; o < 27; ++o) {
      for (int s = 0; s < P.n_st; ++s) {
        int32_t e = P.st_parity[(size_t)p * P.n_st + s];
        int d[3] = {(int8_t)(e & 0xff), (int8_t)((e >> 8) & 0xff), (int8_t)((e >> 16) & 0xff)};
        int so = (floor_div8(loc[0] + d[0]) + 1) + 3 * (floor_div8(loc[1] + d[1]) + 1) +
                 9 * (floor_div8(loc[2] + d[2]) + 1);
        if (so == o) P.cell_ent.push_back(e);
      }
      P.cell_ent_off.push_back((int32_t)P.cell_ent.size());
      cell_cnt[l * 27 + o] = P.cell_ent_off.back() - P.cell_ent_off[P.cell_ent_off.size() - 2];
    }
  }

  // ---------------- work lists ----------------
  P.interior_nodes.clear();
  P.leaf_nodes.clear();
  P.boundary_nodes.clear();
  for (int k = 0; k < n; ++k) {
    if (P.children[8 * k] >= 0) {
      P.interior_nodes.push_back(k);
    } else {
      P.leaf_nodes.push_back(k);
      bool b = false;
      for (int o = 0; o < 27; ++o) {
        int m = P.nbr[27 * k + o];
        if (m >= 0 && P.children[8 * m] >= 0) b = true;
      }
      if (b) P.boundary_nodes.push_back(k);
    }
  }
  P.bnd_index.assign(n, -1);
  P.bnd_perm.assign(P.boundary_nodes.size() * kCells, 0);
  for (size_t bi = 0; bi < P.boundary_nodes.size(); ++bi) {
    const int k = P.boundary_nodes[bi];
    P.bnd_index[k] = (int32_t)bi;
    std::vector<int> load(kCells, 0);
    for (int l = 0; l < kCells; ++l)
      for (int o = 0; o < 27; ++o) {
        const int m = P.nbr[27 * k + o];
        if (m >= 0 && P.children[8 * m] >= 0) load[l] += cell_cnt[l * 27 + o];
      }
    std::vector<int> cells(kCells);
    for (int l = 0; l < kCells; ++l) cells[l] = l;
    std::stable_sort(cells.begin(), cells.end(), [&](int x, int y) { return load[x] > load[y]; });
    for (int i = 0; i < kCells; ++i) P.bnd_perm[bi * kCells + i] = (uint16_t)cells[i];
  }

  // ---------------- same-level counts ----------------
  // Per neighbour slot o: number of (cell, offset) pairs landing in slot o.
  auto slot_of = [](int loc, int d) { return floor_div8(loc + d) + 1; };
  std::vector<int64_t> far_slot(27, 0), near_slot(27, 0);
  for (int c = 0; c < kCells; ++c) {
    int loc[3] = {c & 7, (c >> 3) & 7, c >> 6};
    int p = (loc[0] & 1) + 2 * (loc[1] & 1) + 4 * (loc[2] & 1);
    auto acc = [&](const int32_t* tab, int cnt, std::vector<int64_t>& dst) {
      for (int s = 0; s < cnt; ++s) {
        int32_t e = tab[s];
        int d[3] = {(int8_t)(e & 0xff), (int8_t)((e >> 8) & 0xff), (int8_t)((e >> 16) & 0xff)};
        int o = slot_of(loc[0], d[0]) + 3 * slot_of(loc[1], d[1]) + 9 * slot_of(loc[2], d[2]);
        dst[o] += 1;
      }
    };
    acc(&P.st_parity[(size_t)p * P.n_st], P.n_st, far_slot);
    acc(P.st_near.data(), (int)P.st_near.size(), near_slot);
  }
  int64_t c_m2l = 0, c_p2p = 0;
  int64_t* kp = P.kernel_pairs;
  for (int k = 0; k < n; ++k) {
    bool leaf = P.children[8 * k] < 0;
    if (P.level[k] == 0) {
      for (int c = 0; c < kCells; ++c) {
        int loc[3] = {c & 7, (c >> 3) & 7, c >> 6};
        for (int32_t e : P.st_root) {
          int d[3] = {(int8_t)(e & 0xff), (int8_t)((e >> 8) & 0xff), (int8_t)((e >> 16) & 0xff)};
          bool in = true;
          for (int a = 0; a < 3; ++a) in = in && loc[a] + d[a] >= 0 && loc[a] + d[a] < 8;
          c_m2l += in;
          kp[leaf ? 1 : 0] += in;
        }
        if (leaf)
          for (int32_t e : P.st_near) {
            int d[3] = {(int8_t)(e & 0xff), (int8_t)((e >> 8) & 0xff), (int8_t)((e >> 16) & 0xff)};
            bool in = true;
            for (int a = 0; a < 3; ++a) in = in && loc[a] + d[a] >= 0 && loc[a] + d[a] < 8;
            c_p2p += in;
            kp[2] += in;
          }
      }
      continue;
    }
    for (int o = 0; o < 27; ++o) {
      int m = P.nbr[27 * k + o];
      if (m < 0) continue;
      c_m2l += far_slot[o];
      bool mleaf = P.children[8 * m] < 0;
      kp[!leaf ? 0 : (mleaf ? 1 : 3)] += far_slot[o];
      if (leaf && mleaf) {
        c_p2p += near_slot[o];
        kp[2] += near_slot[o];
      }
    }
  }

  // ---------------- cross-level pairs ----------------
  // A leaf cell A meets a near refined cell B of its own level: the walk splits B
  // (recursively) until each piece is far (M2L) or a leaf cell (P2P).
  struct XPair {
    int64_t tgt, src;
    int kind;  // 0 M2L, 1 P2P
  };
  std::vector<XPair> xp;
  int64_t c_xm2l = 0, c_xp2p = 0;
  struct Cell {
    int node, loc;
    int level;
    int64_t I[3];
  };
  auto cell_children = [&](const Cell& B, Cell out[8]) {
    int la[3] = {B.loc & 7, (B.loc >> 3) & 7, B.loc >> 6};
    int o = (la[0] >> 2) + 2 * (la[1] >> 2) + 4 * (la[2] >> 2);
    int ch = P.children[8 * B.node + o];
    int k = 0;
    for (int ez = 0; ez < 2; ++ez)
      for (int ey = 0; ey < 2; ++ey)
        for (int ex = 0; ex < 2; ++ex) {
          int e[3] = {ex, ey, ez};
          Cell c;
          c.node = ch;
          c.level = B.level + 1;
          int l2[3];
          for (int a = 0; a < 3; ++a) {
            l2[a] = 2 * (la[a] & 3) + e[a];
            c.I[a] = 2 * B.I[a] + e[a];
          }
          c.loc = l2[0] + 8 * l2[1] + 64 * l2[2];
          out[k++] = c;
        }
  };
  std::vector<Cell> stack;
  for (int T : P.boundary_nodes) {
    int lv = P.level[T];
    for (int c = 0; c < kCells; ++c) {
      int loc[3] = {c & 7, (c >> 3) & 7, c >> 6};
      Cell A;
      A.node = T;
      A.loc = c;
      A.level = lv;
      for (int a = 0; a < 3; ++a) A.I[a] = 8 * (int64_t)P.ijk[3 * T + a] + loc[a];
      int64_t gA = (int64_t)T * kCells + c;
      for (int32_t e : P.st_near) {
        int d[3] = {(int8_t)(e & 0xff), (int8_t)((e >> 8) & 0xff), (int8_t)((e >> 16) & 0xff)};
        int o = slot_of(loc[0], d[0]) + 3 * slot_of(loc[1], d[1]) + 9 * slot_of(loc[2], d[2]);
        int N = P.nbr[27 * T + o];
        if (N < 0 || P.children[8 * N] < 0) continue;
        Cell B;
        B.node = N;
        B.level = lv;
        int lb[3];
        for (int a = 0; a < 3; ++a) {
          lb[a] = (loc[a] + d[a]) & 7;
          B.I[a] = A.I[a] + d[a];
        }
        B.loc = lb[0] + 8 * lb[1] + 64 * lb[2];
        stack.clear();
        stack.push_back(B);
        while (!stack.empty()) {
          Cell X = stack.back();
          stack.pop_back();
          Cell ch[8];
          cell_children(X, ch);
          for (int q = 0; q < 8; ++q) {
            const Cell& b = ch[q];
            bool b_leaf = P.children[8 * b.node] < 0;
            bool far = well_separated(theta, A.level, A.I, b.level, b.I);
            if (far || b_leaf) {
              int64_t gb = (int64_t)b.node * kCells + b.loc;
              xp.push_back({gA, gb, far ? 0 : 1});
              xp.push_back({gb, gA, far ? 0 : 1});
              if (far)
                c_xm2l += 2;
              else
                c_xp2p += 2;
            } else {
              stack.push_back(b);
            }
          }
        }
      }
    }
  }
  std::sort(xp.begin(), xp.end(), [](const XPair& a, const XPair& b) {
    if (a.tgt != b.tgt) return a.tgt < b.tgt;
    if (a.kind != b.kind) return a.kind < b.kind;
    return a.src < b.src;
  });
  P.x_targets.clear();
  P.x_start.clear();
  P.x_mid.clear();
  P.x_sources.resize(xp.size());
  for (size_t i = 0; i < xp.size(); ++i) {
    if (i == 0 || xp[i].tgt != xp[i - 1].tgt) {
      P.x_targets.push_back(xp[i].tgt);
      P.x_start.push_back((int64_t)i);
      P.x_mid.push_back(-1);
    }
    if (xp[i].kind == 1 && P.x_mid.back() < 0) P.x_mid.back() = (int64_t)i;
    P.x_sources[i] = xp[i].src;
  }
  P.x_start.push_back((int64_t)xp.size());
  for (size_t t = 0; t < P.x_targets.size(); ++t)
    if (P.x_mid[t] < 0) P.x_mid[t] = P.x_start[t + 1];
  split_cross_pairs(P);

  P.counts[0] = c_m2l;
  P.counts[1] = c_xm2l;
  P.counts[2] = c_p2p;
  P.counts[3] = c_xp2p;
  return OCTO_OK;
}

}  // namespace octo
