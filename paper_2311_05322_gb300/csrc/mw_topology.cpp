// Host topology for lowest-order Nedelec elements (Sec. IV-D) and the subdomains of the
// one-level ORAS preconditioner (Sec. IV-C).  Canonical numbering rules are stated in mw.h.
#include <algorithm>
#include <climits>
#include <cstring>
#include <numeric>

#include "mw_internal.h"

namespace mw {

static const int kLocalEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
// local face k is opposite local vertex k
static const int kLocalFace[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

namespace {

struct FaceKey {
  int32_t a, b, c;   // sorted vertex ids
  int32_t tet;       // owning tet
  int8_t k;          // local face index
  bool operator<(const FaceKey& o) const {
    if (a != o.a) return a < o.a;
    if (b != o.b) return b < o.b;
    if (c != o.c) return c < o.c;
    return tet < o.tet;
  }
  bool same(const FaceKey& o) const { return a == o.a && b == o.b && c == o.c; }
};

inline void sort3(int32_t& a, int32_t& b, int32_t& c) {
  if (a > b) std::swap(a, b);
  if (b > c) std::swap(b, c);
  if (a > b) std::swap(a, b);
}

// Index of edge (lo, hi) given per-vertex sorted neighbour lists.
inline int64_t find_edge(const std::vector<int64_t>& vptr, const std::vector<int32_t>& vhi, int32_t lo, int32_t hi) {
  const int32_t* beg = vhi.data() + vptr[lo];
  const int32_t* end = vhi.data() + vptr[lo + 1];
  const int32_t* it = std::lower_bound(beg, end, hi);
  if (it == end || *it != hi) return -1;
  return (int64_t)(it - vhi.data());
}

}  // namespace

bool build_topology(int64_t n_vert, int64_t n_tet, const int32_t* tv, Topology& t, Error& err) {
  if (n_vert <= 0 || n_tet <= 0 || !tv) {
    err = {MW_EINVAL, "mesh needs n_vert > 0, n_tet > 0 and a tet array"};
    return false;
  }
  if (n_vert > INT32_MAX || 36 * n_tet > INT32_MAX) {
    err = {MW_EINVAL, "mesh too large for 32-bit indices"};
    return false;
  }
  t = Topology();
  t.n_vert = n_vert;
  t.n_tet = n_tet;
  t.tets.assign(tv, tv + 4 * n_tet);
  for (int64_t i = 0; i < 4 * n_tet; ++i) {
    if (tv[i] < 0 || tv[i] >= n_vert) {
      err = {MW_EINVAL, "tet vertex id out of range"};
      return false;
    }
  }
  for (int64_t e = 0; e < n_tet; ++e) {
    const int32_t* v = tv + 4 * e;
    for (int i = 0; i < 4; ++i)
      for (int j = i + 1; j < 4; ++j)
        if (v[i] == v[j]) {
          err = {MW_EINVAL, "tet with repeated vertex"};
          return false;
        }
  }

  // ---- edges: per-lo-vertex sorted unique hi lists; id = lexicographic rank ----
  std::vector<int64_t> vcnt(n_vert + 1, 0);
  for (int64_t e = 0; e < n_tet; ++e)
    for (int l = 0; l < 6; ++l) {
      int32_t a = tv[4 * e + kLocalEdge[l][0]], b = tv[4 * e + kLocalEdge[l][1]];
      vcnt[std::min(a, b) + 1]++;
    }
  for (int64_t v = 0; v < n_vert; ++v) vcnt[v + 1] += vcnt[v];
  std::vector<int32_t> vhi_raw(vcnt[n_vert]);
  {
    std::vector<int64_t> fill(vcnt.begin(), vcnt.end() - 1);
    for (int64_t e = 0; e < n_tet; ++e)
      for (int l = 0; l < 6; ++l) {
        int32_t a = tv[4 * e + kLocalEdge[l][0]], b = tv[4 * e + kLocalEdge[l][1]];
        vhi_raw[fill[std::min(a, b)]++] = std::max(a, b);
      }
  }
  std::vector<int64_t> vptr(n_vert + 1, 0);
  std::vector<int32_t> vhi;
  vhi.reserve(vhi_raw.size() / 2);
  for (int64_t v = 0; v < n_vert; ++v) {
    int32_t* b = vhi_raw.data() + vcnt[v];
    int32_t* e = vhi_raw.data() + vcnt[v + 1];
    std::sort(b, e);
    int32_t* u = std::unique(b, e);
    vhi.insert(vhi.end(), b, u);
    vptr[v + 1] = (int64_t)vhi.size();
  }
  vhi_raw.clear();
  vhi_raw.shrink_to_fit();
  t.n_edge = (int64_t)vhi.size();
  if (t.n_edge > INT32_MAX) {
    err = {MW_EINVAL, "too many edges"};
    return false;
  }
  t.edge_vert.resize(2 * t.n_edge);
  for (int64_t v = 0; v < n_vert; ++v)
    for (int64_t k = vptr[v]; k < vptr[v + 1]; ++k) {
      t.edge_vert[2 * k] = (int32_t)v;
      t.edge_vert[2 * k + 1] = vhi[k];
    }
  t.tet_edge.resize(6 * n_tet);
  t.tet_sign.resize(6 * n_tet);
  for (int64_t e = 0; e < n_tet; ++e)
    for (int l = 0; l < 6; ++l) {
      int32_t a = tv[4 * e + kLocalEdge[l][0]], b = tv[4 * e + kLocalEdge[l][1]];
      t.tet_edge[6 * e + l] = (int32_t)find_edge(vptr, vhi, std::min(a, b), std::max(a, b));
      t.tet_sign[6 * e + l] = a < b ? 1 : -1;
    }

  // ---- CSR pattern: union of the 6 edges of every tet incident to the row edge ----
  const int64_t E = t.n_edge;
  std::vector<int64_t> etp(E + 1, 0);
  for (int64_t i = 0; i < 6 * n_tet; ++i) etp[t.tet_edge[i] + 1]++;
  for (int64_t e = 0; e < E; ++e) etp[e + 1] += etp[e];
  std::vector<int32_t> et(etp[E]);
  {
    std::vector<int64_t> fill(etp.begin(), etp.end() - 1);
    for (int64_t e = 0; e < n_tet; ++e)
      for (int l = 0; l < 6; ++l) et[fill[t.tet_edge[6 * e + l]]++] = (int32_t)e;
  }
  t.row_ptr.assign(E + 1, 0);
  std::vector<int32_t> scratch;
  {
    std::vector<int32_t> cols;
    cols.reserve(36 * n_tet / 2);
    for (int64_t r = 0; r < E; ++r) {
      scratch.clear();
      for (int64_t k = etp[r]; k < etp[r + 1]; ++k) {
        const int32_t* te = t.tet_edge.data() + 6 * (int64_t)et[k];
        scratch.insert(scratch.end(), te, te + 6);
      }
      std::sort(scratch.begin(), scratch.end());
      auto u = std::unique(scratch.begin(), scratch.end());
      cols.insert(cols.end(), scratch.begin(), u);
      t.row_ptr[r + 1] = (int64_t)cols.size();
    }
    t.col_idx.swap(cols);
  }
  t.nnz = (int64_t)t.col_idx.size();
  if (t.nnz > INT32_MAX) {
    err = {MW_EINVAL, "pattern too large"};
    return false;
  }
  auto pos_of = [&](int32_t r, int32_t c) -> int64_t {
    const int32_t* b = t.col_idx.data() + t.row_ptr[r];
    const int32_t* e = t.col_idx.data() + t.row_ptr[r + 1];
    const int32_t* it = std::lower_bound(b, e, c);
    return (int64_t)(it - t.col_idx.data());
  };

  // ---- faces ----
  std::vector<FaceKey> fk(4 * n_tet);
  for (int64_t e = 0; e < n_tet; ++e)
    for (int k = 0; k < 4; ++k) {
      int32_t a = tv[4 * e + kLocalFace[k][0]], b = tv[4 * e + kLocalFace[k][1]], c = tv[4 * e + kLocalFace[k][2]];
      sort3(a, b, c);
      fk[4 * e + k] = {a, b, c, (int32_t)e, (int8_t)k};
    }
  std::sort(fk.begin(), fk.end());
  t.tet_nb.assign(4 * n_tet, -1);
  int64_t nf = 0;
  for (size_t i = 0; i < fk.size();) {
    size_t j = i + 1;
    while (j < fk.size() && fk[j].same(fk[i])) ++j;
    if (j - i > 2) {
      err = {MW_EINVAL, "non-manifold mesh (face shared by more than two tets)"};
      return false;
    }
    if (j - i == 2) {
      t.tet_nb[4 * (int64_t)fk[i].tet + fk[i].k] = fk[i + 1].tet;
      t.tet_nb[4 * (int64_t)fk[i + 1].tet + fk[i + 1].k] = fk[i].tet;
    } else {
      t.bface_vert.push_back(fk[i].a);
      t.bface_vert.push_back(fk[i].b);
      t.bface_vert.push_back(fk[i].c);
    }
    ++nf;
    i = j;
  }
  fk.clear();
  fk.shrink_to_fit();
  t.n_face = nf;
  t.n_bface = (int64_t)t.bface_vert.size() / 3;
  t.bface_edge.resize(3 * t.n_bface);
  for (int64_t f = 0; f < t.n_bface; ++f) {
    const int32_t* q = t.bface_vert.data() + 3 * f;
    t.bface_edge[3 * f + 0] = (int32_t)find_edge(vptr, vhi, q[0], q[1]);
    t.bface_edge[3 * f + 1] = (int32_t)find_edge(vptr, vhi, q[0], q[2]);
    t.bface_edge[3 * f + 2] = (int32_t)find_edge(vptr, vhi, q[1], q[2]);
  }

  // ---- pull map: contributions per nnz, tets in index order then faces in face order ----
  const int64_t n_contrib = 36 * n_tet + 9 * t.n_bface;
  std::vector<int32_t> cpos(n_contrib);
  for (int64_t e = 0; e < n_tet; ++e)
    for (int m = 0; m < 6; ++m)
      for (int n = 0; n < 6; ++n)
        cpos[36 * e + 6 * m + n] = (int32_t)pos_of(t.tet_edge[6 * e + m], t.tet_edge[6 * e + n]);
  for (int64_t f = 0; f < t.n_bface; ++f)
    for (int m = 0; m < 3; ++m)
      for (int n = 0; n < 3; ++n)
        cpos[36 * n_tet + 9 * f + 3 * m + n] = (int32_t)pos_of(t.bface_edge[3 * f + m], t.bface_edge[3 * f + n]);
  t.contrib_ptr.assign(t.nnz + 1, 0);
  for (int64_t i = 0; i < n_contrib; ++i) t.contrib_ptr[cpos[i] + 1]++;
  for (int64_t p = 0; p < t.nnz; ++p) t.contrib_ptr[p + 1] += t.contrib_ptr[p];
  t.contrib.resize(n_contrib);
  {
    std::vector<int64_t> fill(t.contrib_ptr.begin(), t.contrib_ptr.end() - 1);
    for (int64_t i = 0; i < 36 * n_tet; ++i) t.contrib[fill[cpos[i]]++] = (int32_t)i;
    for (int64_t i = 0; i < 9 * t.n_bface; ++i) t.contrib[fill[cpos[36 * n_tet + i]]++] = -(int32_t)i - 1;
  }
  return true;
}

bool build_subdomains(const Topology& t, int32_t n_sub, const int32_t* part, int32_t overlap, Subdomains& sd,
                      Error& err) {
  if (n_sub <= 0 || !part || overlap < 0) {
    err = {MW_EINVAL, "need n_sub > 0, a partition array and overlap >= 0"};
    return false;
  }
  const int64_t T = t.n_tet, E = t.n_edge, V = t.n_vert;
  for (int64_t e = 0; e < T; ++e)
    if (part[e] < 0 || part[e] >= n_sub) {
      err = {MW_EINVAL, "tet_part entry out of [0, n_sub)"};
      return false;
    }
  sd = Subdomains();
  sd.n_sub = n_sub;
  // owner: lowest subdomain id whose own (non-overlapping) tets touch the edge
  sd.owner.assign(E, INT32_MAX);
  for (int64_t e = 0; e < T; ++e)
    for (int l = 0; l < 6; ++l) {
      int32_t& o = sd.owner[t.tet_edge[6 * e + l]];
      o = std::min(o, part[e]);
    }
  // vertex -> tets
  std::vector<int64_t> vtp(V + 1, 0);
  for (int64_t i = 0; i < 4 * T; ++i) vtp[t.tets[i] + 1]++;
  for (int64_t v = 0; v < V; ++v) vtp[v + 1] += vtp[v];
  std::vector<int32_t> vt(vtp[V]);
  {
    std::vector<int64_t> fill(vtp.begin(), vtp.end() - 1);
    for (int64_t e = 0; e < T; ++e)
      for (int k = 0; k < 4; ++k) vt[fill[t.tets[4 * e + k]]++] = (int32_t)e;
  }
  // tets of each subdomain
  std::vector<int64_t> ptp(n_sub + 1, 0);
  for (int64_t e = 0; e < T; ++e) ptp[part[e] + 1]++;
  for (int s = 0; s < n_sub; ++s) ptp[s + 1] += ptp[s];
  std::vector<int32_t> pt(T);
  {
    std::vector<int64_t> fill(ptp.begin(), ptp.end() - 1);
    for (int64_t e = 0; e < T; ++e) pt[fill[part[e]]++] = (int32_t)e;
  }
  std::vector<int32_t> tstamp(T, -1), vstamp(V, -1), estamp(E, -1), eloc(E, 0);
  sd.dof_ptr.assign(1, 0);
  sd.own_ptr.assign(1, 0);
  sd.tet_ptr.assign(1, 0);
  sd.surf_ptr.assign(1, 0);
  std::vector<int32_t> cur, next, dofs;
  for (int32_t s = 0; s < n_sub; ++s) {
    cur.assign(pt.begin() + ptp[s], pt.begin() + ptp[s + 1]);
    for (int32_t e : cur) tstamp[e] = s;
    for (int layer = 0; layer < overlap; ++layer) {
      next.clear();
      for (int32_t e : cur)
        for (int k = 0; k < 4; ++k) {
          int32_t v = t.tets[4 * (int64_t)e + k];
          if (vstamp[v] == s) continue;
          vstamp[v] = s;
          for (int64_t q = vtp[v]; q < vtp[v + 1]; ++q)
            if (tstamp[vt[q]] != s) {
              tstamp[vt[q]] = s;
              next.push_back(vt[q]);
            }
        }
      cur.insert(cur.end(), next.begin(), next.end());
    }
    std::sort(cur.begin(), cur.end());
    dofs.clear();
    for (int32_t e : cur)
      for (int l = 0; l < 6; ++l) {
        int32_t d = t.tet_edge[6 * (int64_t)e + l];
        if (estamp[d] != s) {
          estamp[d] = s;
          dofs.push_back(d);
        }
      }
    std::sort(dofs.begin(), dofs.end());
    for (size_t i = 0; i < dofs.size(); ++i) eloc[dofs[i]] = (int32_t)i;
    for (size_t i = 0; i < dofs.size(); ++i)
      if (sd.owner[dofs[i]] == s) sd.own_local.push_back((int32_t)i);
    sd.dofs.insert(sd.dofs.end(), dofs.begin(), dofs.end());
    for (int32_t e : cur) {
      sd.tet_ids.push_back(e);
      for (int l = 0; l < 6; ++l) sd.tet_loc.push_back(eloc[t.tet_edge[6 * (int64_t)e + l]]);
    }
    // surface faces of the overlapped subdomain: outer boundary (nb < 0) or interface (nb outside)
    for (int32_t e : cur)
      for (int k = 0; k < 4; ++k) {
        int32_t nb = t.tet_nb[4 * (int64_t)e + k];
        if (nb >= 0 && tstamp[nb] == s) continue;
        int32_t q[3] = {t.tets[4 * (int64_t)e + kLocalFace[k][0]], t.tets[4 * (int64_t)e + kLocalFace[k][1]],
                        t.tets[4 * (int64_t)e + kLocalFace[k][2]]};
        sort3(q[0], q[1], q[2]);
        // local dofs of (q0q1, q0q2, q1q2): find among the tet's edges
        int32_t loc[3];
        const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (int p = 0; p < 3; ++p) {
          int32_t lo = q[pairs[p][0]], hi = q[pairs[p][1]];
          loc[p] = -1;
          for (int l = 0; l < 6; ++l) {
            int32_t d = t.tet_edge[6 * (int64_t)e + l];
            if (t.edge_vert[2 * (int64_t)d] == lo && t.edge_vert[2 * (int64_t)d + 1] == hi) loc[p] = eloc[d];
          }
        }
        sd.surf_vert.insert(sd.surf_vert.end(), q, q + 3);
        sd.surf_loc.insert(sd.surf_loc.end(), loc, loc + 3);
        sd.surf_tet.push_back(nb >= 0 ? e : -1);
      }
    sd.dof_ptr.push_back((int64_t)sd.dofs.size());
    sd.own_ptr.push_back((int64_t)sd.own_local.size());
    sd.tet_ptr.push_back((int64_t)sd.tet_ids.size());
    sd.surf_ptr.push_back((int64_t)sd.surf_tet.size());
  }
  return true;
}

namespace {
// Interleaves the low 21 bits of x, y, z (x in the lowest position).
uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  auto spread = [](uint64_t v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
  };
  return spread(x) | (spread(y) << 1) | (spread(z) << 2);
}
}  // namespace

bool build_spmm_plan(const Topology& t, const double* xyz, int halo_max, SpmmPlan& p, Error& err, int row_max,
                     int64_t nnz_max) {
  const int64_t E = t.n_edge;
  if (halo_max < 64 || halo_max > 65535) {
    err = {MW_EINVAL, "halo_max out of range"};
    return false;
  }
  // Morton keys of the edge midpoints on the bounding box
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < t.n_vert; ++v)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], xyz[3 * v + d]);
      hi[d] = std::max(hi[d], xyz[3 * v + d]);
    }
  std::vector<uint64_t> key(E);
  for (int64_t e = 0; e < E; ++e) {
    uint32_t q[3];
    for (int d = 0; d < 3; ++d) {
      const double m = 0.5 * (xyz[3 * (int64_t)t.edge_vert[2 * e] + d] + xyz[3 * (int64_t)t.edge_vert[2 * e + 1] + d]);
      const double u = hi[d] > lo[d] ? (m - lo[d]) / (hi[d] - lo[d]) : 0.0;
      q[d] = (uint32_t)std::min(2097151.0, std::max(0.0, u * 2097151.0));
    }
    key[e] = morton3(q[0], q[1], q[2]);
  }
  std::vector<int32_t> order(E);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  // greedy blocks along that order
  p = SpmmPlan();
  p.rows = order;
  p.blk_row.push_back(0);
  std::vector<int64_t> stamp(E, -1);
  int64_t blk = 0, cnt = 0, nrow = 0, nz = 0;
  for (int64_t i = 0; i < E; ++i) {
    const int32_t r = order[i];
    const int64_t len = t.row_ptr[r + 1] - t.row_ptr[r];
    if (len > nnz_max || len > halo_max) {
      err = {MW_EINVAL, "SpMM plan: a row has more nonzeros than a block holds"};
      return false;
    }
    int64_t fresh = 0;
    for (int64_t k = t.row_ptr[r]; k < t.row_ptr[r + 1]; ++k) fresh += stamp[t.col_idx[k]] != blk;
    if (nrow > 0 && (cnt + fresh > halo_max || nrow + 1 > row_max || nz + len > nnz_max)) {
      p.blk_row.push_back(i);
      ++blk;
      cnt = 0;
      nrow = 0;
      nz = 0;
      fresh = len;
    }
    for (int64_t k = t.row_ptr[r]; k < t.row_ptr[r + 1]; ++k) stamp[t.col_idx[k]] = blk;
    cnt += fresh;
    nz += len;
    ++nrow;
  }
  p.blk_row.push_back(E);
  p.n_block = (int64_t)p.blk_row.size() - 1;
  // halos (ascending), local columns and the value map
  std::vector<int32_t> loc(E, -1);
  p.blk_halo.assign(1, 0);
  p.rptr.assign(1, 0);
  p.lcol.reserve(t.nnz);
  p.src.reserve(t.nnz);
  for (int64_t b = 0; b < p.n_block; ++b) {
    const size_t h0 = p.halo.size();
    for (int64_t i = p.blk_row[b]; i < p.blk_row[b + 1]; ++i) {
      const int32_t r = p.rows[i];
      for (int64_t k = t.row_ptr[r]; k < t.row_ptr[r + 1]; ++k)
        if (loc[t.col_idx[k]] < 0) {
          loc[t.col_idx[k]] = 0;
          p.halo.push_back(t.col_idx[k]);
        }
    }
    std::sort(p.halo.begin() + h0, p.halo.end());
    if (p.halo.size() - h0 > (size_t)halo_max) {
      err = {MW_ECUDA, "SpMM plan: a block's halo exceeds its bound"};
      return false;
    }
    for (size_t j = h0; j < p.halo.size(); ++j) loc[p.halo[j]] = (int32_t)(j - h0);
    for (int64_t i = p.blk_row[b]; i < p.blk_row[b + 1]; ++i) {
      const int32_t r = p.rows[i];
      for (int64_t k = t.row_ptr[r]; k < t.row_ptr[r + 1]; ++k) {
        p.lcol.push_back((uint16_t)loc[t.col_idx[k]]);
        p.src.push_back((int32_t)k);
      }
      p.rptr.push_back((int64_t)p.lcol.size());
    }
    for (size_t j = h0; j < p.halo.size(); ++j) loc[p.halo[j]] = -1;
    p.blk_halo.push_back((int64_t)p.halo.size());
  }
  return true;
}

}  // namespace mw
