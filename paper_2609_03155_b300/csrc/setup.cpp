// dpg_setup_mesh host logic: validation, entity numbering of the trace
// unknowns, Dirichlet values, removal of unpaired H-hat unknowns, element
// colouring and the CSR pattern of the condensed trace system.
//
// Trace unknowns (Sec. 2.3): the tangential trace of the Nedelec space of
// order r = p + 1 keeps the edge functions (r per edge) and face functions
// (2 r (r - 1) per face); interior functions are discarded.  Entities are
// identified by their vertex ids: an edge by (start, end) along the local
// axis, a face by its sorted vertex ids, with the corner order of the first
// element that meets it stored to check that neighbours agree.
//
// Mixed trial degrees: an entity carries trace unknowns of order
// r_E = min over the elements that contain it of (p_K + 1), so that the trace
// lies in every neighbour's own trace space; each element still computes at
// its own degree.  Element K's trace coefficients are the global trace's values
// at K's own nodes, uhat_K = R_K uhat, and R_K's entries are 1D Lagrange
// polynomials of the entity order evaluated at K's nodes (on a face the edge
// unknowns enter through the closed Lagrange factor of the face order at the
// face's two edges).  The global unknowns an element touches sit in its own
// trace slots (same entity, same index) and the slots without one are marked
// unused (-2), so R_K is a square matrix over the element's trace slots.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <unordered_map>

#include "dpg_internal.h"

namespace dpg {

namespace {

struct FaceKeyHash {
  size_t operator()(const std::array<int, 4>& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int v : k) {
      h ^= (uint64_t)(uint32_t)v;
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};

// Trilinear Jacobian J[a][b] = dx_a / dxi_b and position at reference point xi.
void trilinear(const double* X /*8x3*/, const double* xi, double J[3][3], double x[3]) {
  for (int a = 0; a < 3; ++a) {
    x[a] = 0;
    for (int b = 0; b < 3; ++b) J[a][b] = 0;
  }
  for (int v = 0; v < 8; ++v) {
    double f[3], df[3];
    for (int a = 0; a < 3; ++a) {
      int bit = (v >> a) & 1;
      f[a] = bit ? xi[a] : 1.0 - xi[a];
      df[a] = bit ? 1.0 : -1.0;
    }
    double shape = f[0] * f[1] * f[2];
    for (int a = 0; a < 3; ++a) {
      x[a] += shape * X[3 * v + a];
      J[a][0] += df[0] * f[1] * f[2] * X[3 * v + a];
      J[a][1] += f[0] * df[1] * f[2] * X[3 * v + a];
      J[a][2] += f[0] * f[1] * df[2] * X[3 * v + a];
    }
  }
}

double det3(const double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

void inv3(const double J[3][3], double Ji[3][3]) {
  double d = det3(J);
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / d;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / d;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / d;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / d;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / d;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / d;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / d;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / d;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / d;
}

struct cplx {
  double re, im;
};
cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
cplx cexpi(double t) { return {std::cos(t), std::sin(t)}; }
cplx csqrt_(cplx z) {
  double m = std::sqrt(std::hypot(z.re, z.im));
  double th = 0.5 * std::atan2(z.im, z.re);
  return {m * std::cos(th), m * std::sin(th)};
}

// E of the TE_mn mode (Sec. 4.1) at x; H not needed on Dirichlet faces.
void te_E(const dpg_dirichlet_group& g, double omega, const double x[3], cplx E[3]) {
  const double pi = 3.14159265358979323846;
  double k1 = g.m * pi / g.a, k2 = g.n * pi / g.b, kc2 = k1 * k1 + k2 * k2;
  cplx eps{g.eps_re, g.eps_im}, mu{g.mu_re, g.mu_im};
  cplx em = cmul(eps, mu);
  cplx k3 = csqrt_({omega * omega * em.re - kc2, omega * omega * em.im});
  // i k3 x3
  cplx ph = cexpi(k3.re * x[2]);
  double decay = std::exp(-k3.im * x[2]);
  ph.re *= decay;
  ph.im *= decay;
  cplx pre = cmul({0.0, omega}, mu);  // i w mu
  pre.re /= kc2;
  pre.im /= kc2;
  double c1 = std::cos(k1 * x[0]), s1 = std::sin(k1 * x[0]);
  double c2 = std::cos(k2 * x[1]), s2 = std::sin(k2 * x[1]);
  cplx e0 = cmul(pre, {-k2 * c1 * s2, 0.0});
  cplx e1 = cmul(pre, {k1 * s1 * c2, 0.0});
  E[0] = cmul(e0, ph);
  E[1] = cmul(e1, ph);
  E[2] = {0.0, 0.0};
}

}  // namespace

int build_mesh(dpg_handle* h, const dpg_mesh_desc* m, const dpg_params* prm, cudaStream_t s) {
  if (!m || !prm || !m->vert || !m->elem || !m->elem_p || !m->elem_eps || !m->elem_mu || !m->face_bc ||
      !m->face_grp || m->n_vert <= 0 || m->n_elem <= 0) {
    h->err = "null mesh array or empty mesh";
    return DPG_ERR_ARG;
  }
  if (prm->dp != 1) {
    h->err = "only dp = 1 is implemented";
    return DPG_ERR_UNSUPPORTED;
  }
  if (!(prm->alpha > 0) || !(prm->omega > 0)) {
    h->err = "alpha and omega must be positive";
    return DPG_ERR_ARG;
  }
  if (prm->precision < DPG_PREC_FP64 || prm->precision > DPG_PREC_3XTF32) {
    h->err = "unsupported precision mode";
    return DPG_ERR_UNSUPPORTED;
  }
  const int ne = m->n_elem;
  for (int e = 0; e < ne; ++e)
    if (m->elem_p[e] < 1 || m->elem_p[e] > MAXP) {
      h->err = "trial degree must be in 1..4 (element " + std::to_string(e) + ")";
      return DPG_ERR_MESH;
    }
  for (int64_t k = 0; k < (int64_t)ne * 8; ++k)
    if (m->elem[k] < 0 || m->elem[k] >= m->n_vert) {
      h->err = "element vertex id out of range";
      return DPG_ERR_MESH;
    }
  for (int64_t k = 0; k < (int64_t)ne * 6; ++k) {
    int bc = m->face_bc[k], g = m->face_grp[k];
    if (bc == DPG_BC_ROBIN && (g < 0 || g >= m->n_robin || !m->robin)) {
      h->err = "Robin group out of range";
      return DPG_ERR_MESH;
    }
    if (bc == DPG_BC_DIRICHLET && (g < 0 || g >= m->n_dirichlet || !m->dirichlet)) {
      h->err = "Dirichlet group out of range";
      return DPG_ERR_MESH;
    }
    if (bc < 0 || bc > 2) {
      h->err = "face tag out of range";
      return DPG_ERR_MESH;
    }
  }
  h->ne = ne;
  h->prec = prm->precision;
  h->omega = prm->omega;
  h->alpha = prm->alpha;
  h->robin.assign(m->robin, m->robin + m->n_robin);
  h->dirichlet.assign(m->dirichlet, m->dirichlet + m->n_dirichlet);
  // ---- order groups ------------------------------------------------------
  {
    int slot_of_p[MAXP + 1];
    for (int q = 0; q <= MAXP; ++q) slot_of_p[q] = -1;
    for (int e = 0; e < ne; ++e) slot_of_p[m->elem_p[e]] = 0;
    h->grp.clear();
    for (int q = 1; q <= MAXP; ++q)
      if (slot_of_p[q] == 0) {
        slot_of_p[q] = (int)h->grp.size();
        Group G;
        G.p = q;
        G.sz = make_sizes(q);
        build_tables(q, &G.tab);
        h->grp.push_back(std::move(G));
      }
    h->elem_grp.assign(ne, 0);
    for (int e = 0; e < ne; ++e) {
      h->elem_grp[e] = (int8_t)slot_of_p[m->elem_p[e]];
      h->grp[h->elem_grp[e]].elems.push_back(e);
    }
    h->szmax = h->grp.back().sz;
  }
  // ---- geometry: corner coordinates and corner Jacobians ---------------
  std::vector<double> X((size_t)ne * 24);
  for (int e = 0; e < ne; ++e)
    for (int v = 0; v < 8; ++v)
      for (int a = 0; a < 3; ++a) X[(size_t)e * 24 + 3 * v + a] = m->vert[3 * (size_t)m->elem[8 * (size_t)e + v] + a];
  for (int e = 0; e < ne; ++e)
    for (int v = 0; v < 8; ++v) {
      double xi[3] = {double(v & 1), double((v >> 1) & 1), double((v >> 2) & 1)}, J[3][3], x[3];
      trilinear(&X[(size_t)e * 24], xi, J, x);
      if (!(det3(J) > 0)) {
        h->err = "element with non-positive Jacobian at a corner (element " + std::to_string(e) + ")";
        return DPG_ERR_MESH;
      }
    }

  // ---- entities -------------------------------------------------------
  auto corner = [&](int e, int i, int j, int k) { return m->elem[8 * (size_t)e + i + 2 * j + 4 * k]; };
  std::unordered_map<uint64_t, int> edge_id;
  std::unordered_map<std::array<int, 4>, int, FaceKeyHash> face_id;
  std::vector<std::array<int, 4>> face_order;
  std::vector<int> elem_edge((size_t)ne * 12), elem_face((size_t)ne * 6);
  int n_edges = 0, n_faces = 0;
  for (int e = 0; e < ne; ++e) {
    for (int c = 0; c < 3; ++c) {
      int d1 = (c == 0) ? 1 : 0, d2 = (c == 2) ? 1 : 2;
      for (int s2 = 0; s2 < 2; ++s2)
        for (int s1 = 0; s1 < 2; ++s1) {
          int pos[3];
          pos[d1] = s1;
          pos[d2] = s2;
          pos[c] = 0;
          int v0 = corner(e, pos[0], pos[1], pos[2]);
          pos[c] = 1;
          int v1 = corner(e, pos[0], pos[1], pos[2]);
          uint64_t key = ((uint64_t)(uint32_t)v0 << 32) | (uint32_t)v1;
          uint64_t rkey = ((uint64_t)(uint32_t)v1 << 32) | (uint32_t)v0;
          if (edge_id.count(rkey)) {
            h->err = "edge orientation differs between neighbours (element " + std::to_string(e) + ")";
            return DPG_ERR_MESH;
          }
          auto it = edge_id.find(key);
          int id;
          if (it == edge_id.end()) {
            id = n_edges++;
            edge_id.emplace(key, id);
          } else {
            id = it->second;
          }
          elem_edge[(size_t)e * 12 + c * 4 + s1 + 2 * s2] = id;
        }
    }
    for (int d = 0; d < 3; ++d)
      for (int sd = 0; sd < 2; ++sd) {
        int a = (d == 0) ? 1 : 0, b = (d == 2) ? 1 : 2;
        std::array<int, 4> ord;
        int k = 0;
        for (int tb = 0; tb < 2; ++tb)
          for (int ta = 0; ta < 2; ++ta) {
            int pos[3];
            pos[d] = sd;
            pos[a] = ta;
            pos[b] = tb;
            ord[k++] = corner(e, pos[0], pos[1], pos[2]);
          }
        std::array<int, 4> key = ord;
        std::sort(key.begin(), key.end());
        auto it = face_id.find(key);
        int id;
        if (it == face_id.end()) {
          id = n_faces++;
          face_id.emplace(key, id);
          face_order.push_back(ord);
        } else {
          id = it->second;
          if (face_order[id] != ord) {
            h->err = "face orientation differs between neighbours (element " + std::to_string(e) + ")";
            return DPG_ERR_MESH;
          }
        }
        elem_face[(size_t)e * 6 + 2 * d + sd] = id;
      }
  }
  const int n_ent = n_edges + n_faces;  // entity id: edges [0, n_edges), faces after
  // entity trace order: min over the containing elements of p + 1
  std::vector<int> ent_r(n_ent, MAXP + 1);
  for (int e = 0; e < ne; ++e) {
    const int re = m->elem_p[e] + 1;
    for (int k = 0; k < 12; ++k) ent_r[elem_edge[(size_t)e * 12 + k]] = std::min(ent_r[elem_edge[(size_t)e * 12 + k]], re);
    for (int k = 0; k < 6; ++k)
      ent_r[n_edges + elem_face[(size_t)e * 6 + k]] = std::min(ent_r[n_edges + elem_face[(size_t)e * 6 + k]], re);
  }
  auto ent_dofs = [&](int ent) { return ent < n_edges ? ent_r[ent] : 2 * ent_r[ent] * (ent_r[ent] - 1); };

  // ---- boundary classification ------------------------------------------
  // Dirichlet: every entity on a Dirichlet face; data groups win over zero groups.
  std::vector<int> dir_grp(n_ent, -1);            // Dirichlet group deciding the values
  std::vector<int> dir_src_elem(n_ent, -1), dir_src_face(n_ent, -1);
  std::vector<int> face_adj(n_ent, 0), face_robin(n_ent, 0);  // edges: incident element faces
  std::vector<char> face_is_robin(n_faces, 0);
  for (int e = 0; e < ne; ++e)
    for (int f = 0; f < 6; ++f) {
      int d = f / 2, sd = f % 2;
      int bc = m->face_bc[6 * (size_t)e + f], g = m->face_grp[6 * (size_t)e + f];
      // edges of this element face: edges along the two tangential axes with the
      // transverse coordinate d fixed to sd
      int ents[5];
      int k = 0;
      ents[k++] = n_edges + elem_face[(size_t)e * 6 + f];
      for (int c = 0; c < 3; ++c) {
        if (c == d) continue;
        int d1 = (c == 0) ? 1 : 0, d2 = (c == 2) ? 1 : 2;
        for (int s2 = 0; s2 < 2; ++s2)
          for (int s1 = 0; s1 < 2; ++s1) {
            int pos1 = (d1 == d) ? sd : -1, pos2 = (d2 == d) ? sd : -1;
            if ((pos1 >= 0 && s1 != pos1) || (pos2 >= 0 && s2 != pos2)) continue;
            ents[k++] = elem_edge[(size_t)e * 12 + c * 4 + s1 + 2 * s2];
          }
      }
      for (int q = 1; q < k; ++q) {
        face_adj[ents[q]] += 1;
        if (bc == DPG_BC_ROBIN) face_robin[ents[q]] += 1;
      }
      if (bc == DPG_BC_ROBIN) face_is_robin[elem_face[(size_t)e * 6 + f]] = 1;
      if (bc == DPG_BC_DIRICHLET) {
        bool data = h->dirichlet[g].kind != DPG_DIRICHLET_ZERO;
        for (int q = 0; q < k; ++q) {
          int en = ents[q];
          bool take = dir_grp[en] < 0 || (data && h->dirichlet[dir_grp[en]].kind == DPG_DIRICHLET_ZERO);
          if (take) {
            dir_grp[en] = g;
            dir_src_elem[en] = e;
            dir_src_face[en] = f;
          }
        }
      }
    }
  // H-hat unknowns that pair with nothing: faces on Gamma_R, and edges all of
  // whose incident element faces lie on Gamma_R.
  std::vector<char> h_drop(n_ent, 0);
  for (int f = 0; f < n_faces; ++f) h_drop[n_edges + f] = face_is_robin[f];
  for (int ed = 0; ed < n_edges; ++ed) h_drop[ed] = (face_adj[ed] > 0 && face_robin[ed] == face_adj[ed]);

  // ---- global numbering of the free trace unknowns ------------------------
  // Entity-major: each entity's free E-hat unknowns, then its free H-hat
  // unknowns, so the rows of one entity are contiguous and share one column list.
  std::vector<int64_t> startE(n_ent, -1), startH(n_ent, -1);
  int64_t nfree = 0;
  for (int en = 0; en < n_ent; ++en) {
    if (dir_grp[en] < 0) {
      startE[en] = nfree;
      nfree += ent_dofs(en);
    }
    if (!h_drop[en]) {
      startH[en] = nfree;
      nfree += ent_dofs(en);
    }
  }
  if (nfree >= (int64_t)1 << 31) {
    h->err = "more than 2^31 trace unknowns";
    return DPG_ERR_UNSUPPORTED;
  }
  h->n = nfree;

  // ---- element-local map, per-element offsets, trace restrictions ----------
  // Per group: for each local trace function its element entity slot (edges
  // 0..11, faces 12..17) and its (component, open index, closed index), and
  // the inverse lookup (slot, within-entity index at the group's order) -> t.
  struct LocalMap {
    std::vector<int> pk, ent, c, ia, ib, idx;  // ib: closed index along the face's other axis (faces)
    std::vector<std::vector<int>> lookup;  // [slot][within-entity index] -> t
  };
  std::vector<LocalMap> lmap(h->grp.size());
  for (size_t gi = 0; gi < h->grp.size(); ++gi) {
    const int r = h->grp[gi].sz.r, nt = h->grp[gi].sz.nt;
    const std::vector<int> trf = trace_functions(r);
    LocalMap& L = lmap[gi];
    L.pk = trf;
    L.ent.resize(nt);
    L.c.resize(nt);
    L.ia.resize(nt);
    L.ib.resize(nt);
    L.idx.resize(nt);
    L.lookup.assign(18, std::vector<int>(2 * r * r, -1));
    for (int t = 0; t < nt; ++t) {
      int pk = trf[t];
      int c = pk & 3, ii[3] = {(pk >> 2) & 15, (pk >> 6) & 15, (pk >> 10) & 15};
      int d1 = (c == 0) ? 1 : 0, d2 = (c == 2) ? 1 : 2;
      bool b1 = ii[d1] == 0 || ii[d1] == r, b2 = ii[d2] == 0 || ii[d2] == r;
      L.c[t] = c;
      L.ia[t] = ii[c];
      if (b1 && b2) {
        L.ent[t] = c * 4 + (ii[d1] == r) + 2 * (ii[d2] == r);  // element edge slot 0..11
        L.idx[t] = ii[c];
        L.ib[t] = -1;
      } else {
        int dn = b1 ? d1 : d2;  // face normal
        int sd = ii[dn] == r;
        int a = (dn == 0) ? 1 : 0, b = (dn == 2) ? 1 : 2;
        int eo = (c == a) ? b : a;  // other tangential axis
        L.ent[t] = 12 + 2 * dn + sd;
        L.ib[t] = ii[eo];
        L.idx[t] = (c == a ? 0 : 1) * r * (r - 1) + ii[c] * (r - 1) + (ii[eo] - 1);
      }
      L.lookup[L.ent[t]][L.idx[t]] = t;
    }
  }
  auto elem_entity = [&](int e, int slot) {
    return slot < 12 ? elem_edge[(size_t)e * 12 + slot] : n_edges + elem_face[(size_t)e * 6 + slot - 12];
  };
  // offsets into the pooled stores
  h->off.assign(ne + 1, ElemOff{0, 0, 0, 0, 0});
  for (int e = 0; e < ne; ++e) {
    const Sizes& Z = h->grp[h->elem_grp[e]].sz;
    ElemOff o = h->off[e];
    o.S += (int64_t)Z.n_h * Z.n_h;
    o.Z += (int64_t)Z.n_u * Z.n_h;
    o.L1 += (int64_t)Z.n_u * Z.n_u;
    o.h += Z.n_h;
    o.u += Z.n_u;
    h->off[e + 1] = o;
  }
  const ElemOff tot = h->off[ne];
  h->l2g.assign((size_t)tot.h, -2);
  std::vector<double2> xfix((size_t)tot.h, make_double2(0.0, 0.0));
  h->elem_sig.assign(ne, -1);
  h->rsig.clear();
  std::vector<int32_t> rint;
  std::vector<double> rdbl;
  std::map<std::vector<int>, int> sig_id;
  for (int e = 0; e < ne; ++e) {
    const Group& G = h->grp[h->elem_grp[e]];
    const LocalMap& L = lmap[h->elem_grp[e]];
    const int r = G.sz.r, nt = G.sz.nt;
    const int64_t o = h->off[e].h;
    double onode[MAXF1D], cnode[MAXF1D], wdum[MAXF1D];
    bool restricted = false;
    for (int t = 0; t < nt; ++t) {
      const int en = elem_entity(e, L.ent[t]);
      const int rE = ent_r[en];
      if (rE < r) restricted = true;
      int q;  // index within the entity at its own order, or -1 (slot unused)
      if (L.ent[t] < 12) {
        q = L.ia[t] < rE ? L.ia[t] : -1;
      } else {
        const int comp = L.idx[t] / (r * (r - 1));
        q = (L.ia[t] < rE && L.ib[t] <= rE - 1) ? comp * rE * (rE - 1) + L.ia[t] * (rE - 1) + (L.ib[t] - 1) : -1;
      }
      if (q < 0) continue;
      int32_t gE = dir_grp[en] >= 0 ? -1 : (int32_t)(startE[en] + q);
      int32_t gH = h_drop[en] ? -2 : (int32_t)(startH[en] + q);
      h->l2g[o + t] = gE;
      h->l2g[o + nt + t] = gH;
      if (gE == -1) {
        const dpg_dirichlet_group& g = h->dirichlet[dir_grp[en]];
        double2 val = make_double2(0.0, 0.0);
        if (g.kind != DPG_DIRICHLET_ZERO) {
          // nodal interpolation at the entity's own nodes: open node q of
          // order rE along c, closed nodes of order rE across (the element's
          // corner coordinates 0 / 1 on the entity); evaluated in this element
          // (the node and J e_c agree between neighbours)
          gauss_legendre01(rE, onode, wdum);
          gauss_lobatto01(rE + 1, cnode);
          const int pk = L.pk[t];
          const int c = pk & 3, ii[3] = {(pk >> 2) & 15, (pk >> 6) & 15, (pk >> 10) & 15};
          double xi[3];
          for (int d = 0; d < 3; ++d) {
            if (d == c)
              xi[d] = onode[L.ia[t]];
            else
              xi[d] = ii[d] == 0 ? 0.0 : (ii[d] == r ? 1.0 : cnode[ii[d]]);
          }
          double J[3][3], x[3];
          trilinear(&X[(size_t)e * 24], xi, J, x);
          // outward unit normal of the deciding Dirichlet face, at its centre
          // (boundary faces are planar; the datum n x E_D refers to it)
          int f = dir_src_face[en], es = dir_src_elem[en];
          int d = f / 2;
          double xc[3] = {0.5, 0.5, 0.5}, Js[3][3], xs[3], Jsi[3][3];
          xc[d] = (f % 2) ? 1.0 : 0.0;
          trilinear(&X[(size_t)es * 24], xc, Js, xs);
          inv3(Js, Jsi);
          double sgn = (f % 2) ? 1.0 : -1.0;
          double nrm[3] = {sgn * Jsi[d][0], sgn * Jsi[d][1], sgn * Jsi[d][2]};
          double nn = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
          for (int a = 0; a < 3; ++a) nrm[a] /= nn;
          cplx Et[3];
          if (g.kind == DPG_DIRICHLET_SIN_PI_X2) {
            // n x E = v with v = (sin(pi x2), 0, 0)  =>  E_t = v x n
            double v[3] = {std::sin(3.14159265358979323846 * x[1]), 0.0, 0.0};
            Et[0] = {v[1] * nrm[2] - v[2] * nrm[1], 0.0};
            Et[1] = {v[2] * nrm[0] - v[0] * nrm[2], 0.0};
            Et[2] = {v[0] * nrm[1] - v[1] * nrm[0], 0.0};
          } else {
            cplx E[3];
            te_E(g, h->omega, x, E);
            // E_t = E - (E . n) n
            cplx en_{0, 0};
            for (int a = 0; a < 3; ++a) {
              en_.re += E[a].re * nrm[a];
              en_.im += E[a].im * nrm[a];
            }
            for (int a = 0; a < 3; ++a) Et[a] = {E[a].re - en_.re * nrm[a], E[a].im - en_.im * nrm[a]};
          }
          for (int a = 0; a < 3; ++a) {
            val.x += Et[a].re * J[a][c];
            val.y += Et[a].im * J[a][c];
          }
        }
        xfix[o + t] = val;
      }
    }
    if (!restricted) continue;
    // signature: degree and the orders of the 18 entities
    std::vector<int> key(19);
    key[0] = r;
    for (int k = 0; k < 18; ++k) key[1 + k] = ent_r[elem_entity(e, k)];
    auto it = sig_id.find(key);
    if (it != sig_id.end()) {
      h->elem_sig[e] = it->second;
      continue;
    }
    // R (nt x nt, one field): row t = element trace function, column = slot
    std::vector<double> R((size_t)nt * nt, 0.0);
    double oK[MAXF1D], cK[MAXF1D];
    gauss_legendre01(r, oK, wdum);
    gauss_lobatto01(r + 1, cK);
    double val[MAXF1D], der[MAXF1D], vo[MAXF1D], vc[MAXF1D];
    for (int t = 0; t < nt; ++t) {
      const int slot = L.ent[t];
      const int c = L.c[t];
      const double xc = oK[L.ia[t]];
      auto add_edge = [&](int eslot, double scale) {
        const int re = key[1 + eslot];
        double on[MAXF1D];
        gauss_legendre01(re, on, wdum);
        lagrange1d(on, re, xc, val, der);
        for (int q = 0; q < re; ++q) {
          const int col = L.lookup[eslot][q];
          R[(size_t)t * nt + col] += scale * val[q];
        }
      };
      if (slot < 12) {
        add_edge(slot, 1.0);
        continue;
      }
      const int rF = key[1 + slot];
      const int dn = (slot - 12) / 2, sd = (slot - 12) % 2;
      const int a = (dn == 0) ? 1 : 0, b = (dn == 2) ? 1 : 2;
      const int eo = (c == a) ? b : a;
      const int comp = (c == a) ? 0 : 1;
      const double xe = cK[L.ib[t]];
      double on[MAXF1D], cn[MAXF1D];
      gauss_legendre01(rF, on, wdum);
      gauss_lobatto01(rF + 1, cn);
      lagrange1d(on, rF, xc, vo, der);
      lagrange1d(cn, rF + 1, xe, vc, der);
      for (int ia = 0; ia < rF; ++ia)
        for (int ib = 1; ib < rF; ++ib) {
          const int col = L.lookup[slot][comp * r * (r - 1) + ia * (r - 1) + (ib - 1)];
          R[(size_t)t * nt + col] += vo[ia] * vc[ib];
        }
      // the face's two edges along c, at eo = 0 (closed end 0) and eo = 1 (end rF)
      for (int send = 0; send < 2; ++send) {
        int pos[3];
        pos[dn] = sd;
        pos[eo] = send;
        const int d1 = (c == 0) ? 1 : 0, d2 = (c == 2) ? 1 : 2;
        const int eslot = c * 4 + pos[d1] + 2 * pos[d2];
        add_edge(eslot, vc[send ? rF : 0]);
      }
    }
    RSig rs{};
    rs.nt = nt;
    rs.cptr = (int64_t)rint.size();
    std::vector<int> cnt(nt + 1, 0);
    for (int t = 0; t < nt; ++t)
      for (int col = 0; col < nt; ++col)
        if (R[(size_t)t * nt + col] != 0.0) cnt[col + 1]++;
    for (int col = 0; col < nt; ++col) cnt[col + 1] += cnt[col];
    rint.insert(rint.end(), cnt.begin(), cnt.end());
    rs.cidx = (int64_t)rint.size();
    rs.cw = (int64_t)rdbl.size();
    for (int col = 0; col < nt; ++col)
      for (int t = 0; t < nt; ++t)
        if (R[(size_t)t * nt + col] != 0.0) {
          rint.push_back(t);
          rdbl.push_back(R[(size_t)t * nt + col]);
        }
    rs.rptr = (int64_t)rint.size();
    std::vector<int> rc(nt + 1, 0);
    for (int t = 0; t < nt; ++t)
      for (int col = 0; col < nt; ++col)
        if (R[(size_t)t * nt + col] != 0.0) rc[t + 1]++;
    for (int t = 0; t < nt; ++t) rc[t + 1] += rc[t];
    rint.insert(rint.end(), rc.begin(), rc.end());
    rs.ridx = (int64_t)rint.size();
    rs.rw = (int64_t)rdbl.size();
    for (int t = 0; t < nt; ++t)
      for (int col = 0; col < nt; ++col)
        if (R[(size_t)t * nt + col] != 0.0) {
          rint.push_back(col);
          rdbl.push_back(R[(size_t)t * nt + col]);
        }
    const int id = (int)h->rsig.size();
    h->rsig.push_back(rs);
    sig_id.emplace(key, id);
    h->elem_sig[e] = id;
  }

  // ---- colouring (elements sharing a vertex get different colours) ----------
  {
    std::vector<std::vector<int>> v2e(m->n_vert);
    for (int e = 0; e < ne; ++e)
      for (int v = 0; v < 8; ++v) v2e[m->elem[8 * (size_t)e + v]].push_back(e);
    std::vector<int> color(ne, -1);
    int ncol = 0;
    std::vector<int> mark;
    for (int e = 0; e < ne; ++e) {
      mark.assign(ncol + 1, 0);
      for (int v = 0; v < 8; ++v)
        for (int o : v2e[m->elem[8 * (size_t)e + v]])
          if (color[o] >= 0) mark[color[o]] = 1;
      int c = 0;
      while (c < ncol && mark[c]) ++c;
      color[e] = c;
      if (c == ncol) ++ncol;
    }
    // per group: its elements sorted by colour
    h->ncolor = ncol;
    for (Group& G : h->grp) {
      G.color_off.assign(ncol + 1, 0);
      for (int e : G.elems) G.color_off[color[e] + 1]++;
      for (int c = 0; c < ncol; ++c) G.color_off[c + 1] += G.color_off[c];
      G.color_elems_host.assign(G.elems.size(), 0);
      std::vector<int> fill(G.color_off.begin(), G.color_off.end() - 1);
      for (int e : G.elems) G.color_elems_host[fill[color[e]]++] = e;
    }
  }

  // ---- CSR pattern: the rows of one entity share their column list ----------
  // Row i of entity block b has its W_b values at rowptr[i] and its columns
  // in cols[colptr_b .. colptr_b + W_b) (sorted).  Only these per-entity lists
  // are stored, not one column index per non-zero.
  std::vector<std::vector<int>> ent_elems(n_ent);
  for (int e = 0; e < ne; ++e) {
    for (int k = 0; k < 12; ++k) ent_elems[elem_edge[(size_t)e * 12 + k]].push_back(e);
    for (int k = 0; k < 6; ++k) ent_elems[n_edges + elem_face[(size_t)e * 6 + k]].push_back(e);
  }
  h->blk.clear();
  h->blk_colptr.clear();
  h->cols.clear();
  std::vector<int64_t> rowptr(nfree + 1, 0);
  std::vector<int32_t> row2blk(nfree, -1);
  for (int en = 0; en < n_ent; ++en) {
    const int dE = startE[en] >= 0 ? ent_dofs(en) : 0, dH = startH[en] >= 0 ? ent_dofs(en) : 0;
    if (dE + dH == 0) continue;
    std::vector<int> nb;
    for (int e : ent_elems[en]) {
      for (int k = 0; k < 12; ++k) nb.push_back(elem_edge[(size_t)e * 12 + k]);
      for (int k = 0; k < 6; ++k) nb.push_back(n_edges + elem_face[(size_t)e * 6 + k]);
    }
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    const int64_t cp = (int64_t)h->cols.size();
    int W = 0;
    for (int o : nb) {  // entity-major numbering: neighbours in entity order give sorted columns
      if (startE[o] >= 0)
        for (int k = 0; k < ent_dofs(o); ++k) h->cols.push_back((int32_t)(startE[o] + k));
      if (startH[o] >= 0)
        for (int k = 0; k < ent_dofs(o); ++k) h->cols.push_back((int32_t)(startH[o] + k));
    }
    W = (int)((int64_t)h->cols.size() - cp);
    const int64_t row0 = dE ? startE[en] : startH[en];
    const int b = (int)h->blk.size();
    h->blk.push_back({(int)row0, dE + dH, W, 0});
    h->blk_colptr.push_back(cp);
    for (int k = 0; k < dE + dH; ++k) row2blk[row0 + k] = b;
  }
  for (int64_t i = 0; i < nfree; ++i) rowptr[i + 1] = rowptr[i] + h->blk[row2blk[i]].z;
  h->nnz = rowptr[nfree];
  h->nblk = (int)h->blk.size();
  h->blk_dmax = 0;
  for (const int4& B : h->blk) h->blk_dmax = std::max(h->blk_dmax, B.y);
  // diagonal position of each block's own unknowns inside its column list
  for (int b = 0; b < h->nblk; ++b) {
    const int4& B = h->blk[b];
    const int32_t* c = &h->cols[h->blk_colptr[b]];
    int pos = 0;
    while (pos < B.z && c[pos] != B.x) ++pos;
    h->blk[b].w = pos;
  }

  // ---- element classes: lossless elements without a Robin face are real ----
  h->is_real.assign(ne, 0);
  for (int e = 0; e < ne; ++e) {
    bool real = m->elem_eps[e].im == 0.0 && m->elem_mu[e].im == 0.0;
    for (int f = 0; f < 6; ++f)
      if (m->face_bc[6 * (size_t)e + f] == DPG_BC_ROBIN) real = false;
    h->is_real[e] = real;
  }
  h->eps_host.assign(m->elem_eps, m->elem_eps + ne);
  h->mu_host.assign(m->elem_mu, m->elem_mu + ne);
  h->robin_face.assign(ne, 0);
  for (int e = 0; e < ne; ++e)
    for (int f = 0; f < 6; ++f)
      if (m->face_bc[6 * (size_t)e + f] == DPG_BC_ROBIN) h->robin_face[e] = 1;
  classify_elements(h);

  // ---- Robin entries ---------------------------------------------------------
  h->robin_entries.clear();
  h->robin_first.assign(ne, -1);
  for (int e = 0; e < ne; ++e)
    for (int f = 0; f < 6; ++f)
      if (m->face_bc[6 * (size_t)e + f] == DPG_BC_ROBIN) {
        if (h->robin_first[e] < 0) h->robin_first[e] = (int)h->robin_entries.size();
        h->robin_entries.push_back({e, f, m->face_grp[6 * (size_t)e + f]});
      }

  // ---- device buffers --------------------------------------------------------
  auto alloc = [&](void** ptr, size_t bytes) -> int {
    if (bytes == 0) bytes = 16;
    cudaError_t er = cudaMalloc(ptr, bytes);
    if (er != cudaSuccess) {
      h->err = std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(er);
      cudaGetLastError();
      return DPG_ERR_NOMEM;
    }
    return DPG_OK;
  };
#define DPG_ALLOC(ptr, bytes)                                  \
  do {                                                         \
    int rc_ = alloc((void**)&(ptr), (size_t)(bytes));          \
    if (rc_) return rc_;                                       \
  } while (0)
  DPG_ALLOC(h->d_X, sizeof(double) * 24 * (size_t)ne);
  DPG_ALLOC(h->d_eps, sizeof(double2) * ne);
  DPG_ALLOC(h->d_mu, sizeof(double2) * ne);
  DPG_ALLOC(h->d_fbc, 6 * (size_t)ne);
  DPG_ALLOC(h->d_off, sizeof(ElemOff) * (ne + 1));
  DPG_ALLOC(h->d_l2g, sizeof(int32_t) * tot.h);
  DPG_ALLOC(h->d_xfix, sizeof(double2) * tot.h);
  DPG_ALLOC(h->d_robin, sizeof(dpg_robin_group) * std::max<size_t>(1, h->robin.size()));
  DPG_ALLOC(h->d_status, sizeof(int) * (ne + 1));  // [ne]: tensor-core wait timeout flag
  DPG_ALLOC(h->d_S, sizeof(double2) * tot.S);
  DPG_ALLOC(h->d_s, sizeof(double2) * tot.h);
  DPG_ALLOC(h->d_c, sizeof(double) * ne);
  DPG_ALLOC(h->d_Z, sizeof(double2) * tot.Z);
  DPG_ALLOC(h->d_z, sizeof(double2) * tot.u);
  if (prm->flags & DPG_FLAG_ADJOINT) DPG_ALLOC(h->d_L1, sizeof(double2) * tot.L1);
  DPG_ALLOC(h->d_sig, sizeof(int) * ne);
  DPG_ALLOC(h->d_rsig, sizeof(RSig) * std::max<size_t>(1, h->rsig.size()));
  DPG_ALLOC(h->d_rint, sizeof(int32_t) * std::max<size_t>(1, rint.size()));
  DPG_ALLOC(h->d_rdbl, sizeof(double) * std::max<size_t>(1, rdbl.size()));
  DPG_ALLOC(h->d_rowptr, sizeof(int64_t) * (nfree + 1));
  DPG_ALLOC(h->d_row2blk, sizeof(int32_t) * nfree);
  DPG_ALLOC(h->d_blk, sizeof(int4) * h->nblk);
  DPG_ALLOC(h->d_blk_colptr, sizeof(int64_t) * h->nblk);
  DPG_ALLOC(h->d_cols, sizeof(int32_t) * h->cols.size());
  DPG_ALLOC(h->d_val, sizeof(double2) * h->nnz);
  DPG_ALLOC(h->d_b, sizeof(double2) * nfree);
  for (Group& G : h->grp) {
    const Sizes& Z = G.sz;
    DPG_ALLOC(G.d_trfun, sizeof(int) * Z.nt);
    DPG_ALLOC(G.d_Xref, sizeof(double) * Z.n_f * Z.n_f);
    DPG_ALLOC(G.d_Tf, sizeof(double) * 6 * Z.n_f * Z.nt);
    DPG_ALLOC(G.d_Tall, sizeof(double) * Z.n_f * Z.nt);
    DPG_ALLOC(G.d_elems, sizeof(int) * G.elems.size());
    DPG_ALLOC(G.d_color_elems, sizeof(int) * G.elems.size());
  }
#undef DPG_ALLOC
  std::vector<double2> eps(ne), mu(ne);
  for (int e = 0; e < ne; ++e) {
    eps[e] = make_double2(m->elem_eps[e].re, m->elem_eps[e].im);
    mu[e] = make_double2(m->elem_mu[e].re, m->elem_mu[e].im);
  }
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_X, X.data(), sizeof(double) * X.size(), cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_eps, eps.data(), sizeof(double2) * ne, cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_mu, mu.data(), sizeof(double2) * ne, cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_fbc, m->face_bc, 6 * (size_t)ne, cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_off, h->off.data(), sizeof(ElemOff) * (ne + 1), cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_l2g, h->l2g.data(), sizeof(int32_t) * h->l2g.size(), cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_xfix, xfix.data(), sizeof(double2) * xfix.size(), cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_sig, h->elem_sig.data(), sizeof(int) * ne, cudaMemcpyHostToDevice, s));
  if (!h->rsig.empty()) {
    DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_rsig, h->rsig.data(), sizeof(RSig) * h->rsig.size(), cudaMemcpyHostToDevice, s));
    DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_rint, rint.data(), sizeof(int32_t) * rint.size(), cudaMemcpyHostToDevice, s));
    DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_rdbl, rdbl.data(), sizeof(double) * rdbl.size(), cudaMemcpyHostToDevice, s));
  }
  for (Group& G : h->grp) {
    const std::vector<int> trf = trace_functions(G.sz.r);
    DPG_CUDA_TRY(h, cudaMemcpyAsync(G.d_trfun, trf.data(), sizeof(int) * trf.size(), cudaMemcpyHostToDevice, s));
    DPG_CUDA_TRY(h, cudaMemcpyAsync(G.d_elems, G.elems.data(), sizeof(int) * G.elems.size(), cudaMemcpyHostToDevice, s));
    DPG_CUDA_TRY(h, cudaMemcpyAsync(G.d_color_elems, G.color_elems_host.data(), sizeof(int) * G.elems.size(),
                                    cudaMemcpyHostToDevice, s));
    // the per-group host vector trf dies here: wait for its copy
    DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  }
  if (!h->robin.empty())
    DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_robin, h->robin.data(), sizeof(dpg_robin_group) * h->robin.size(),
                                    cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_rowptr, rowptr.data(), sizeof(int64_t) * rowptr.size(), cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_row2blk, row2blk.data(), sizeof(int32_t) * nfree, cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_blk, h->blk.data(), sizeof(int4) * h->nblk, cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_blk_colptr, h->blk_colptr.data(), sizeof(int64_t) * h->nblk,
                                  cudaMemcpyHostToDevice, s));
  DPG_CUDA_TRY(h, cudaMemcpyAsync(h->d_cols, h->cols.data(), sizeof(int32_t) * h->cols.size(), cudaMemcpyHostToDevice,
                                  s));
  DPG_CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int) * (ne + 1), s));
  // the host vectors above die at return: wait for the copies
  DPG_CUDA_TRY(h, cudaStreamSynchronize(s));
  return DPG_OK;
}

// Split every group's elements into lossless (real path) and the others.
void classify_elements(dpg_handle* h) {
  for (Group& G : h->grp) {
    G.real_elems.clear();
    G.cplx_elems.clear();
    for (int e : G.elems) (h->is_real[e] ? G.real_elems : G.cplx_elems).push_back(e);
  }
}

}  // namespace dpg
