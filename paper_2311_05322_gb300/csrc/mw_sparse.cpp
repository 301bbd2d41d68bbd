// Symbolic multifrontal factorisation of the ORAS subdomain matrices (host side).
//
// Each subdomain's dofs (edges) are ordered by geometric nested dissection: a set larger than
// the leaf size is split at the median of its edge midpoints along its longest extent, and the
// dofs of the lower half that share a tet with the upper half form the separator.  The
// separator is eliminated after both halves, so the tree's post-order is the elimination order.
// A node's update set holds the later-eliminated dofs coupled to its pivots, directly or through
// a descendant's update set; its front is [pivots (padded to a multiple of 32) | update dofs].
#include <algorithm>
#include <numeric>

#include "mw_internal.h"

namespace mw {
namespace {

struct Tree {
  std::vector<std::vector<int32_t>> piv;   // pivots of each node (post-order ids)
  std::vector<std::vector<int32_t>> kids;
};

struct NdBuilder {
  const std::vector<int64_t>& adj_ptr;
  const std::vector<int32_t>& adj;
  const std::vector<double>& co;   // [n][3] edge midpoints
  int leaf;
  std::vector<int32_t> side;       // tag of the upper half during a split
  int32_t tag = 0;
  Tree t;

  int32_t build(std::vector<int32_t> ids) {
    if ((int)ids.size() <= leaf) {
      std::sort(ids.begin(), ids.end());
      t.piv.push_back(std::move(ids));
      t.kids.push_back({});
      return (int32_t)t.piv.size() - 1;
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int32_t i : ids)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], co[3 * (size_t)i + d]);
        hi[d] = std::max(hi[d], co[3 * (size_t)i + d]);
      }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    const size_t half = ids.size() / 2;
    std::nth_element(ids.begin(), ids.begin() + half, ids.end(), [&](int32_t a, int32_t b) {
      const double ca = co[3 * (size_t)a + ax], cb = co[3 * (size_t)b + ax];
      return ca != cb ? ca < cb : a < b;
    });
    std::vector<int32_t> left(ids.begin(), ids.begin() + half), right(ids.begin() + half, ids.end());
    ids.clear();
    ids.shrink_to_fit();
    const int32_t tg = ++tag;
    for (int32_t j : right) side[j] = tg;
    std::vector<int32_t> sep, rest;
    for (int32_t i : left) {
      bool cut = false;
      for (int64_t q = adj_ptr[i]; q < adj_ptr[i + 1] && !cut; ++q) cut = side[adj[q]] == tg;
      (cut ? sep : rest).push_back(i);
    }
    std::vector<int32_t> ch;
    if (!rest.empty()) ch.push_back(build(std::move(rest)));
    if (!right.empty()) ch.push_back(build(std::move(right)));
    std::sort(sep.begin(), sep.end());
    t.piv.push_back(std::move(sep));
    t.kids.push_back(std::move(ch));
    return (int32_t)t.piv.size() - 1;
  }
};

}  // namespace

bool build_multifrontal(const Topology& t, const Subdomains& sd, const std::vector<double>& xyz,
                        const uint8_t* metal, int leaf, Multifrontal& mf, Error& err) {
  mf = Multifrontal();
  const int P = Multifrontal::kPad;
  mf.sub_node_ptr.assign(1, 0);
  mf.piv_ptr.assign(1, 0);
  mf.upd_ptr.assign(1, 0);
  mf.child_ptr.assign(1, 0);
  mf.asm_ptr.assign(1, 0);
  mf.asm_sub_ptr.assign(1, 0);
  int64_t fac = 0;
  for (int s = 0; s < sd.n_sub; ++s) {
    const int64_t d0 = sd.dof_ptr[s], n = sd.dof_ptr[s + 1] - d0;
    const int32_t* dof = sd.dofs.data() + d0;
    // local adjacency: dofs sharing a tet
    std::vector<std::vector<int32_t>> nb(n);
    for (int64_t q = sd.tet_ptr[s]; q < sd.tet_ptr[s + 1]; ++q) {
      const int32_t* l = &sd.tet_loc[6 * q];
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b)
          if (a != b) nb[l[a]].push_back(l[b]);
    }
    std::vector<int64_t> adj_ptr(n + 1, 0);
    std::vector<int32_t> adj;
    for (int64_t i = 0; i < n; ++i) {
      std::sort(nb[i].begin(), nb[i].end());
      nb[i].erase(std::unique(nb[i].begin(), nb[i].end()), nb[i].end());
      adj.insert(adj.end(), nb[i].begin(), nb[i].end());
      adj_ptr[i + 1] = (int64_t)adj.size();
      std::vector<int32_t>().swap(nb[i]);
    }
    std::vector<double> co(3 * n);
    for (int64_t i = 0; i < n; ++i) {
      const int32_t e = dof[i];
      const int32_t a = t.edge_vert[2 * (int64_t)e], b = t.edge_vert[2 * (int64_t)e + 1];
      for (int d = 0; d < 3; ++d) co[3 * i + d] = 0.5 * (xyz[3 * (int64_t)a + d] + xyz[3 * (int64_t)b + d]);
    }
    NdBuilder nd{adj_ptr, adj, co, std::max(leaf, 1), std::vector<int32_t>(n, 0), 0, {}};
    std::vector<int32_t> all(n);
    std::iota(all.begin(), all.end(), 0);
    nd.build(std::move(all));
    Tree& tr = nd.t;
    const int32_t nn = (int32_t)tr.piv.size();
    const int32_t base = mf.n_nodes;
    // elimination rank and owning node of every dof
    std::vector<int64_t> rank(n), first(nn), last(nn);
    std::vector<int32_t> owner(n), ppos(n);
    int64_t r = 0;
    for (int32_t k = 0; k < nn; ++k) {
      first[k] = r;
      for (size_t i = 0; i < tr.piv[k].size(); ++i) {
        const int32_t d = tr.piv[k][i];
        rank[d] = r++;
        owner[d] = k;
        ppos[d] = (int32_t)i;
      }
      last[k] = r;
    }
    if (r != n) {
      err = {MW_EINVAL, "nested dissection lost a dof"};
      return false;
    }
    // update sets, bottom-up (post-order)
    std::vector<std::vector<int32_t>> upd(nn);
    std::vector<int32_t> mark(n, -1);
    std::vector<int32_t> par(nn, -1);
    for (int32_t k = 0; k < nn; ++k)
      for (int32_t c : tr.kids[k]) par[c] = k;
    for (int32_t k = 0; k < nn; ++k) {
      std::vector<int32_t>& U = upd[k];
      auto add = [&](int32_t j) {
        if (rank[j] >= last[k] && mark[j] != k) {
          mark[j] = k;
          U.push_back(j);
        }
      };
      for (int32_t i : tr.piv[k])
        for (int64_t q = adj_ptr[i]; q < adj_ptr[i + 1]; ++q) add(adj[q]);
      for (int32_t c : tr.kids[k])
        for (int32_t j : upd[c]) add(j);
      std::sort(U.begin(), U.end(), [&](int32_t a, int32_t b) { return rank[a] < rank[b]; });
    }
    // heights
    std::vector<int32_t> hgt(nn, 0);
    for (int32_t k = 0; k < nn; ++k)
      for (int32_t c : tr.kids[k]) hgt[k] = std::max(hgt[k], hgt[c] + 1);
    // node tables and workspace layout
    std::vector<int64_t> wso(nn);
    int64_t ws = 0;
    for (int32_t k = 0; k < nn; ++k) {
      const int32_t pr = (int32_t)tr.piv[k].size();
      const int32_t pp = (pr + P - 1) / P * P;
      const int32_t uu = (int32_t)upd[k].size();
      const int64_t ff = (int64_t)pp + uu;
      mf.sub.push_back(s);
      mf.p.push_back(pp);
      mf.preal.push_back(pr);
      mf.u.push_back(uu);
      mf.f.push_back(ff);
      mf.height.push_back(hgt[k]);
      mf.parent.push_back(par[k] < 0 ? -1 : base + par[k]);
      mf.fac_off.push_back(fac);
      fac += (int64_t)pp * ff + (int64_t)uu * pp;
      mf.piv_loc.insert(mf.piv_loc.end(), tr.piv[k].begin(), tr.piv[k].end());
      mf.piv_ptr.push_back((int64_t)mf.piv_loc.size());
      mf.upd_loc.insert(mf.upd_loc.end(), upd[k].begin(), upd[k].end());
      mf.upd_ptr.push_back((int64_t)mf.upd_loc.size());
      for (int32_t c : tr.kids[k]) mf.child.push_back(base + c);
      mf.child_ptr.push_back((int64_t)mf.child.size());
      mf.max_height = std::max(mf.max_height, hgt[k]);
      wso[k] = ws;
      mf.ws_off.push_back(ws);
      ws += ff * ff;
    }
    mf.ws_size.push_back(ws);
    // position of dof d in node k's front: pivot row, or p_k + its index in the update set
    auto front_row = [&](int32_t k, int32_t d) -> int64_t {
      if (owner[d] == k) return ppos[d];
      const std::vector<int32_t>& U = upd[k];
      auto it = std::lower_bound(U.begin(), U.end(), d, [&](int32_t a, int32_t b) { return rank[a] < rank[b]; });
      if (it == U.end() || *it != d) return -1;
      return mf.p[base + k] + (int64_t)(it - U.begin());
    };
    // maps from each child's update set into its parent's front rows (indexed by parent row)
    mf.inv_off.resize(base + nn, -1);
    for (int32_t k = 0; k < nn; ++k)
      for (int32_t c : tr.kids[k]) {
        const int64_t ff = mf.f[base + k];
        mf.inv_off[base + c] = (int64_t)mf.inv.size();
        mf.inv.resize(mf.inv.size() + ff, -1);
        int32_t* m = mf.inv.data() + mf.inv_off[base + c];
        for (size_t i = 0; i < upd[c].size(); ++i) {
          const int64_t row = front_row(k, upd[c][i]);
          if (row < 0) {
            err = {MW_EINVAL, "update dof missing from the parent front"};
            return false;
          }
          m[row] = (int32_t)i;
        }
      }
    // original entries -> (node front entry, code)
    auto is_metal = [&](int32_t d) { return metal && metal[dof[d]]; };
    std::vector<std::pair<int64_t, int32_t>> con;
    auto put = [&](int32_t a, int32_t b, int32_t code) -> bool {
      const int32_t k = rank[a] <= rank[b] ? owner[a] : owner[b];
      const int64_t ra = front_row(k, a), rb = front_row(k, b);
      if (ra < 0 || rb < 0) return false;
      con.push_back({wso[k] + ra * mf.f[base + k] + rb, code});
      return true;
    };
    bool ok = true;
    for (int64_t q = sd.tet_ptr[s]; q < sd.tet_ptr[s + 1] && ok; ++q) {
      const int32_t* l = &sd.tet_loc[6 * q];
      for (int a = 0; a < 6 && ok; ++a)
        for (int b = 0; b < 6 && ok; ++b)
          if (!is_metal(l[a]) && !is_metal(l[b])) ok = put(l[a], l[b], (int32_t)(q * 36 + a * 6 + b));
    }
    for (int64_t q = sd.surf_ptr[s]; q < sd.surf_ptr[s + 1] && ok; ++q) {
      const int32_t* l = &sd.surf_loc[3 * q];
      for (int a = 0; a < 3 && ok; ++a)
        for (int b = 0; b < 3 && ok; ++b)
          if (!is_metal(l[a]) && !is_metal(l[b])) ok = put(l[a], l[b], -1 - (int32_t)(q * 9 + a * 3 + b));
    }
    if (!ok) {
      err = {MW_EINVAL, "an element entry falls outside its front"};
      return false;
    }
    for (int64_t d = 0; d < n; ++d)
      if (is_metal((int32_t)d)) put((int32_t)d, (int32_t)d, Multifrontal::kIdentity);
    for (int32_t k = 0; k < nn; ++k)
      for (int32_t i = mf.preal[base + k]; i < mf.p[base + k]; ++i)
        con.push_back({wso[k] + (int64_t)i * mf.f[base + k] + i, Multifrontal::kIdentity});
    std::stable_sort(con.begin(), con.end(),
                     [](const auto& x, const auto& y) { return x.first < y.first; });
    for (size_t i = 0; i < con.size(); ++i) {
      if (i == 0 || con[i].first != con[i - 1].first) {
        if (i) mf.asm_ptr.push_back((int64_t)mf.asm_code.size());
        mf.asm_target.push_back(con[i].first);
      }
      mf.asm_code.push_back(con[i].second);
    }
    if (!con.empty()) mf.asm_ptr.push_back((int64_t)mf.asm_code.size());
    mf.asm_sub_ptr.push_back((int64_t)mf.asm_target.size());
    mf.sub_node_ptr.push_back(base + nn);
    mf.n_nodes = base + nn;
  }
  mf.fac_total = fac;
  return true;
}

}  // namespace mw
