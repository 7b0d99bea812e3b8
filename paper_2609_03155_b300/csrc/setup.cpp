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
#include <functional>
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
  if (!std::isfinite(prm->omega) || !std::isfinite(prm->alpha)) {
    h->err = "omega and alpha must be finite";
    return DPG_ERR_ARG;
  }
  for (int64_t k = 0; k < (int64_t)m->n_vert * 3; ++k)
    if (!std::isfinite(m->vert[k])) {
      h->err = "non-finite vertex coordinate";
      return DPG_ERR_MESH;
    }
  for (int e = 0; e < ne; ++e)
    if (!std::isfinite(m->elem_eps[e].re) || !std::isfinite(m->elem_eps[e].im) || !std::isfinite(m->elem_mu[e].re) ||
        !std::isfinite(m->elem_mu[e].im)) {
      h->err = "non-finite permittivity or permeability (element " + std::to_string(e) + ")";
      return DPG_ERR_ARG;
    }
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
  // ---- 2:1 hanging entities ---------------------------------------------------
  // A face met by one element only and not on a tagged boundary whose four
  // quarters (corner, two mid-edge points, centre) are faces of other elements
  // is a master; the quarters and the four interior half-lines (mid-edge point
  // to centre) are its slaves.  An edge whose two halves are edges of other
  // elements is the master of the halves.  Points are matched by coordinates.
  std::vector<int> master(n_ent);
  for (int en = 0; en < n_ent; ++en) master[en] = en;
  std::vector<int> owner_elem(n_ent, -1), owner_slot(n_ent, -1);
  for (int e = 0; e < ne; ++e) {
    for (int k = 0; k < 12; ++k) {
      const int en = elem_edge[(size_t)e * 12 + k];
      if (owner_elem[en] < 0) owner_elem[en] = e, owner_slot[en] = k;
    }
    for (int k = 0; k < 6; ++k) {
      const int en = n_edges + elem_face[(size_t)e * 6 + k];
      if (owner_elem[en] < 0) owner_elem[en] = e, owner_slot[en] = 12 + k;
    }
  }
  {
    double span = 0.0;
    for (int64_t k = 0; k < (int64_t)m->n_vert * 3; ++k) span = std::max(span, std::fabs(m->vert[k]));
    const double qscale = 1.0 / (1e-9 * std::max(span, 1e-300));
    auto qkey = [&](const double* x) {
      uint64_t hsh = 1469598103934665603ull;
      for (int a2 = 0; a2 < 3; ++a2) {
        hsh ^= (uint64_t)(int64_t)std::llround(x[a2] * qscale);
        hsh *= 1099511628211ull;
      }
      return hsh;
    };
    std::unordered_map<uint64_t, int> vat;
    for (int v = 0; v < m->n_vert; ++v) vat.emplace(qkey(&m->vert[3 * (size_t)v]), v);
    auto vert_at = [&](const double* x) {
      auto it = vat.find(qkey(x));
      if (it == vat.end()) return -1;
      const double* y = &m->vert[3 * (size_t)it->second];
      for (int a2 = 0; a2 < 3; ++a2)
        if (std::fabs(y[a2] - x[a2]) > 1e-8 * std::max(span, 1e-300)) return -1;
      return it->second;
    };
    auto mid = [&](int v0, int v1, double* out) {
      for (int a2 = 0; a2 < 3; ++a2) out[a2] = 0.5 * (m->vert[3 * (size_t)v0 + a2] + m->vert[3 * (size_t)v1 + a2]);
    };
    auto find_edge = [&](int v0, int v1) {
      auto it = edge_id.find(((uint64_t)(uint32_t)v0 << 32) | (uint32_t)v1);
      if (it != edge_id.end()) return it->second;
      it = edge_id.find(((uint64_t)(uint32_t)v1 << 32) | (uint32_t)v0);
      return it == edge_id.end() ? -1 : it->second;
    };
    std::vector<int> face_elems(n_faces, 0);
    std::vector<char> face_tagged(n_faces, 0);
    for (int e = 0; e < ne; ++e)
      for (int k = 0; k < 6; ++k) {
        face_elems[elem_face[(size_t)e * 6 + k]]++;
        if (m->face_bc[6 * (size_t)e + k] != DPG_BC_NONE) face_tagged[elem_face[(size_t)e * 6 + k]] = 1;
      }
    for (int f = 0; f < n_faces; ++f) {
      if (face_elems[f] != 1 || face_tagged[f]) continue;
      const std::array<int, 4>& o = face_order[f];  // corners (0,0), (1,0), (0,1), (1,1)
      double x01[3], x02[3], x13[3], x23[3], xc[3];
      mid(o[0], o[1], x01);
      mid(o[0], o[2], x02);
      mid(o[1], o[3], x13);
      mid(o[2], o[3], x23);
      mid(o[0], o[3], xc);
      const int m01 = vert_at(x01), m02 = vert_at(x02), m13 = vert_at(x13), m23 = vert_at(x23), mc = vert_at(xc);
      if (m01 < 0 || m02 < 0 || m13 < 0 || m23 < 0 || mc < 0) continue;
      const std::array<int, 4> quarters[4] = {{o[0], m01, m02, mc}, {m01, o[1], mc, m13}, {m02, mc, o[2], m23},
                                               {mc, m13, m23, o[3]}};
      int qid[4];
      bool ok = true;
      for (int q = 0; q < 4 && ok; ++q) {
        std::array<int, 4> key = quarters[q];
        std::sort(key.begin(), key.end());
        auto it = face_id.find(key);
        ok = it != face_id.end() && face_elems[it->second] == 1 && !face_tagged[it->second];
        if (ok) qid[q] = it->second;
      }
      const int cross[4] = {find_edge(m01, mc), find_edge(m02, mc), find_edge(mc, m13), find_edge(mc, m23)};
      for (int q = 0; q < 4 && ok; ++q) ok = cross[q] >= 0;
      if (!ok) continue;
      for (int q = 0; q < 4; ++q) {
        master[n_edges + qid[q]] = n_edges + f;
        master[cross[q]] = n_edges + f;
      }
    }
    for (const auto& kv : edge_id) {
      const int v0 = (int)(kv.first >> 32), v1 = (int)(kv.first & 0xffffffffu);
      double xm[3];
      mid(v0, v1, xm);
      const int vm = vert_at(xm);
      if (vm < 0) continue;
      const int h0 = find_edge(v0, vm), h1 = find_edge(vm, v1);
      if (h0 < 0 || h1 < 0) continue;
      master[h0] = kv.second;
      master[h1] = kv.second;
    }
    for (int en = 0; en < n_ent; ++en) {  // follow chains to the top master
      int mm = master[en];
      for (int guard = 0; master[mm] != mm && guard < 8; ++guard) mm = master[mm];
      master[en] = mm;
    }
  }
  h->n_slaves = 0;
  for (int en = 0; en < n_ent; ++en) h->n_slaves += master[en] != en;
  // entity trace order: min over the elements that touch the entity or one of
  // its slaves of p + 1; an edge of a face is capped by the face's order
  std::vector<int> ent_r(n_ent, MAXP + 1);
  for (int e = 0; e < ne; ++e) {
    const int re = m->elem_p[e] + 1;
    for (int k = 0; k < 12; ++k) {
      const int mm = master[elem_edge[(size_t)e * 12 + k]];
      ent_r[mm] = std::min(ent_r[mm], re);
    }
    for (int k = 0; k < 6; ++k) {
      const int mm = master[n_edges + elem_face[(size_t)e * 6 + k]];
      ent_r[mm] = std::min(ent_r[mm], re);
    }
  }
  for (int f = 0; f < n_faces; ++f) {
    const int en = n_edges + f;
    if (master[en] != en) continue;
    const int e = owner_elem[en], kf = owner_slot[en] - 12, d = kf / 2, sd = kf % 2;
    for (int c = 0; c < 3; ++c) {
      if (c == d) continue;
      const int d1 = (c == 0) ? 1 : 0, d2 = (c == 2) ? 1 : 2;
      for (int s2 = 0; s2 < 2; ++s2)
        for (int s1 = 0; s1 < 2; ++s1) {
          if ((d1 == d && s1 != sd) || (d2 == d && s2 != sd)) continue;
          const int mm = master[elem_edge[(size_t)e * 12 + c * 4 + s1 + 2 * s2]];
          ent_r[mm] = std::min(ent_r[mm], ent_r[en]);
        }
    }
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
    if (master[en] != en) continue;  // slaves carry no unknowns
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

  // 1D node sets of every order (open: Gauss-Legendre, closed: Gauss-Lobatto)
  double onodes[MAXF1D][MAXF1D], cnodes[MAXF1D][MAXF1D + 1];
  for (int r = 1; r <= MAXP + 1; ++r) {
    double wd[MAXF1D];
    gauss_legendre01(r, onodes[r], wd);
    gauss_lobatto01(r + 1, cnodes[r]);
  }
  auto lag_open = [&](int r, double x, double* v) {
    double der[MAXF1D + 1];
    lagrange1d(onodes[r], r, x, v, der);
  };
  auto lag_closed = [&](int r, double x, double* v) {
    double der[MAXF1D + 1];
    lagrange1d(cnodes[r], r + 1, x, v, der);
  };
  // reference point of physical x in element e (Newton on the trilinear map)
  auto invert = [&](int e, const double* x, double* xi) {
    xi[0] = xi[1] = xi[2] = 0.5;
    for (int it = 0; it < 30; ++it) {
      double J[3][3], y[3], Ji[3][3];
      trilinear(&X[(size_t)e * 24], xi, J, y);
      inv3(J, Ji);
      double dx[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]}, step = 0.0;
      for (int a2 = 0; a2 < 3; ++a2) {
        const double dxi = Ji[a2][0] * dx[0] + Ji[a2][1] * dx[1] + Ji[a2][2] * dx[2];
        xi[a2] -= dxi;
        step = std::max(step, std::fabs(dxi));
      }
      if (step < 1e-15) break;
    }
  };
  // Trace coefficient along element e's axis c at its reference point xi, on
  // its edge slot ks / face slot kf: terms (global entity, index, weight).  A
  // master entity contributes its own nodal basis (a face also its edges'
  // functions through the closed factor of the face order); a slave is its
  // master's trace at the same physical point times the tangent ratio.
  struct Term {
    int ent, idx;
    double w;
  };
  std::function<void(int, int, const double*, double, std::vector<Term>&)> eval_edge;
  std::function<void(int, int, int, const double*, double, std::vector<Term>&)> eval_face;
  auto eval_master = [&](int M, int e, const double* xi, int c, double scale, std::vector<Term>& out) {
    double J[3][3], x[3], Jm[3][3], xm[3], xim[3];
    trilinear(&X[(size_t)e * 24], xi, J, x);
    const int em = owner_elem[M];
    invert(em, x, xim);
    trilinear(&X[(size_t)em * 24], xim, Jm, xm);
    double tt = 0.0, mm = 0.0;
    for (int a2 = 0; a2 < 3; ++a2) {
      tt += J[a2][c] * Jm[a2][c];
      mm += Jm[a2][c] * Jm[a2][c];
    }
    const double ratio = tt / mm;
    if (M < n_edges)
      eval_edge(em, owner_slot[M], xim, scale * ratio, out);
    else
      eval_face(em, owner_slot[M], c, xim, scale * ratio, out);
  };
  eval_edge = [&](int e, int ks, const double* xi, double scale, std::vector<Term>& out) {
    const int en = elem_edge[(size_t)e * 12 + ks], c = ks / 4;
    if (master[en] != en) {
      eval_master(master[en], e, xi, c, scale, out);
      return;
    }
    const int r = ent_r[en];
    double v[MAXF1D + 1];
    lag_open(r, xi[c], v);
    for (int q = 0; q < r; ++q) out.push_back({en, q, scale * v[q]});
  };
  eval_face = [&](int e, int kf, int c, const double* xi, double scale, std::vector<Term>& out) {
    const int en = n_edges + elem_face[(size_t)e * 6 + kf - 12];
    if (master[en] != en) {
      eval_master(master[en], e, xi, c, scale, out);
      return;
    }
    const int d = (kf - 12) / 2, sd = (kf - 12) % 2;
    const int a = (d == 0) ? 1 : 0, b = (d == 2) ? 1 : 2;
    const int eax = (c == a) ? b : a, comp = (c == a) ? 0 : 1;
    const int rF = ent_r[en];
    double vo[MAXF1D + 1], vc[MAXF1D + 1];
    lag_open(rF, xi[c], vo);
    lag_closed(rF, xi[eax], vc);
    for (int ia = 0; ia < rF; ++ia)
      for (int ib = 1; ib < rF; ++ib)
        out.push_back({en, comp * rF * (rF - 1) + ia * (rF - 1) + (ib - 1), scale * vo[ia] * vc[ib]});
    for (int send = 0; send < 2; ++send) {
      const double wv = vc[send ? rF : 0];
      if (wv == 0.0) continue;
      int pos[3];
      pos[d] = sd;
      pos[eax] = send;
      const int d1 = (c == 0) ? 1 : 0, d2 = (c == 2) ? 1 : 2;
      double xe[3] = {xi[0], xi[1], xi[2]};
      xe[eax] = (double)send;
      eval_edge(e, c * 4 + pos[d1] + 2 * pos[d2], xe, scale * wv, out);
    }
  };

  // Fixed E-hat values per master entity on Dirichlet faces: nodal
  // interpolation of the tangential datum at the entity's own nodes, evaluated
  // in its owner element: coefficient = E_t(x_node) . (J e_c).
  std::vector<std::vector<double2>> fixval(n_ent);
  for (int en = 0; en < n_ent; ++en) {
    if (master[en] != en || dir_grp[en] < 0) continue;
    const dpg_dirichlet_group& g = h->dirichlet[dir_grp[en]];
    const int rE = ent_r[en], nd = ent_dofs(en);
    fixval[en].assign(nd, make_double2(0.0, 0.0));
    if (g.kind == DPG_DIRICHLET_ZERO) continue;
    const int e = owner_elem[en], slot = owner_slot[en];
    for (int q = 0; q < nd; ++q) {
      double xi[3];
      int c;
      if (slot < 12) {
        c = slot / 4;
        const int d1 = (c == 0) ? 1 : 0, d2 = (c == 2) ? 1 : 2;
        xi[c] = onodes[rE][q];
        xi[d1] = (double)((slot % 4) & 1);
        xi[d2] = (double)((slot % 4) >> 1);
      } else {
        const int d = (slot - 12) / 2, sd = (slot - 12) % 2;
        const int a = (d == 0) ? 1 : 0, b = (d == 2) ? 1 : 2;
        const int comp = q / (rE * (rE - 1)), rem = q % (rE * (rE - 1));
        c = comp ? b : a;
        const int eax = comp ? a : b;
        xi[d] = (double)sd;
        xi[c] = onodes[rE][rem / (rE - 1)];
        xi[eax] = cnodes[rE][rem % (rE - 1) + 1];
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
      for (int a2 = 0; a2 < 3; ++a2) nrm[a2] /= nn;
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
        for (int a2 = 0; a2 < 3; ++a2) {
          en_.re += E[a2].re * nrm[a2];
          en_.im += E[a2].im * nrm[a2];
        }
        for (int a2 = 0; a2 < 3; ++a2) Et[a2] = {E[a2].re - en_.re * nrm[a2], E[a2].im - en_.im * nrm[a2]};
      }
      double2 val = make_double2(0.0, 0.0);
      for (int a2 = 0; a2 < 3; ++a2) {
        val.x += Et[a2].re * J[a2][c];
        val.y += Et[a2].im * J[a2][c];
      }
      fixval[en][q] = val;
    }
  }

  // Per element: R rows through the masters, the global entities they touch
  // (elem_ents, which also drive the CSR pattern and the colouring), and a
  // layout of those entities' unknowns in the element's own trace slots.
  h->l2g.assign((size_t)tot.h, -2);
  std::vector<double2> xfix((size_t)tot.h, make_double2(0.0, 0.0));
  h->elem_sig.assign(ne, -1);
  h->rsig.clear();
  std::vector<int32_t> rint;
  std::vector<double> rdbl;
  std::unordered_map<uint64_t, std::vector<int>> sig_by_hash;
  std::vector<std::vector<int>> elem_ents(ne);
  std::vector<Term> terms;
  for (int e = 0; e < ne; ++e) {
    const Group& G = h->grp[h->elem_grp[e]];
    const LocalMap& L = lmap[h->elem_grp[e]];
    const int r = G.sz.r, nt = G.sz.nt;
    const int64_t o = h->off[e].h;
    std::vector<std::vector<Term>> rows(nt);
    for (int t = 0; t < nt; ++t) {
      const int pk = L.pk[t];
      const int c = pk & 3, ii[3] = {(pk >> 2) & 15, (pk >> 6) & 15, (pk >> 10) & 15};
      double xi[3];
      for (int d = 0; d < 3; ++d) xi[d] = d == c ? onodes[r][ii[d]] : cnodes[r][ii[d]];
      terms.clear();
      if (L.ent[t] < 12)
        eval_edge(e, L.ent[t], xi, 1.0, terms);
      else
        eval_face(e, L.ent[t], c, xi, 1.0, terms);
      std::vector<Term>& row = rows[t];
      for (const Term& tm : terms) {  // merge repeated (entity, index)
        if (tm.w == 0.0) continue;
        bool merged = false;
        for (Term& q : row)
          if (q.ent == tm.ent && q.idx == tm.idx) {
            q.w += tm.w;
            merged = true;
            break;
          }
        if (!merged) row.push_back(tm);
      }
    }
    // global entities touched
    std::vector<int>& ge = elem_ents[e];
    for (const auto& row : rows)
      for (const Term& q : row) ge.push_back(q.ent);
    std::sort(ge.begin(), ge.end());
    ge.erase(std::unique(ge.begin(), ge.end()), ge.end());
    // slots: an entity goes to the local slot whose own master it is, the rest
    // to free local slots of the same kind and enough capacity
    int slot_ent[18];
    for (int k = 0; k < 18; ++k) slot_ent[k] = -1;
    std::vector<char> placed(ge.size(), 0);
    for (int k = 0; k < 18; ++k) {
      const int mk = master[elem_entity(e, k)];
      for (size_t gi = 0; gi < ge.size(); ++gi)
        if (!placed[gi] && ge[gi] == mk && ((k < 12) == (mk < n_edges))) {
          slot_ent[k] = mk;
          placed[gi] = 1;
          break;
        }
    }
    for (size_t gi = 0; gi < ge.size(); ++gi) {
      if (placed[gi]) continue;
      const bool is_edge = ge[gi] < n_edges;
      for (int k = is_edge ? 0 : 12; k < (is_edge ? 12 : 18); ++k)
        if (slot_ent[k] < 0 && ent_r[ge[gi]] <= r) {
          slot_ent[k] = ge[gi];
          placed[gi] = 1;
          break;
        }
      if (!placed[gi]) {
        h->err = "element " + std::to_string(e) + ": its constrained trace needs more slots than it has";
        return DPG_ERR_UNSUPPORTED;
      }
    }
    // (entity, global index) -> local trace function t
    auto slot_of = [&](int en, int idx) -> int {
      for (int k = 0; k < 18; ++k)
        if (slot_ent[k] == en) {
          const int rE = ent_r[en];
          if (k < 12) return L.lookup[k][idx];
          const int comp = idx / (rE * (rE - 1)), rem = idx % (rE * (rE - 1));
          return L.lookup[k][comp * r * (r - 1) + (rem / (rE - 1)) * (r - 1) + rem % (rE - 1)];
        }
      return -1;
    };
    // trace map and fixed values of the slots
    for (int k = 0; k < 18; ++k) {
      const int en = slot_ent[k];
      if (en < 0) continue;
      for (int q = 0; q < ent_dofs(en); ++q) {
        const int t = slot_of(en, q);
        const int32_t gE = dir_grp[en] >= 0 ? -1 : (int32_t)(startE[en] + q);
        const int32_t gH = h_drop[en] ? -2 : (int32_t)(startH[en] + q);
        h->l2g[o + t] = gE;
        h->l2g[o + nt + t] = gH;
        if (gE == -1) xfix[o + t] = fixval[en][q];
      }
    }
    // R over the slots: identity for an element whose entities are its own
    // masters at its own order
    std::vector<int> rc(nt + 1, 0), rcol;
    std::vector<double> rw;
    bool identity = true;
    for (int t = 0; t < nt; ++t) {
      for (const Term& q : rows[t]) {
        const int col = slot_of(q.ent, q.idx);
        if (col < 0) {
          h->err = "element " + std::to_string(e) + ": a constrained trace unknown has no slot";
          return DPG_ERR_UNSUPPORTED;
        }
        rcol.push_back(col);
        rw.push_back(q.w);
        identity = identity && col == t && q.w == 1.0;
      }
      rc[t + 1] = (int)rcol.size();
      identity = identity && rows[t].size() == 1;
    }
    if (identity) continue;
    // signature: content hash of the row-compressed R
    uint64_t hsh = 1469598103934665603ull ^ (uint64_t)nt;
    auto mix = [&](uint64_t v) {
      hsh ^= v;
      hsh *= 1099511628211ull;
    };
    for (int t = 0; t <= nt; ++t) mix((uint64_t)rc[t]);
    for (size_t k = 0; k < rcol.size(); ++k) {
      uint64_t bits;
      std::memcpy(&bits, &rw[k], 8);
      mix((uint64_t)rcol[k]);
      mix(bits);
    }
    int found = -1;
    for (int id : sig_by_hash[hsh]) {
      const RSig& q = h->rsig[id];
      if (q.nt != nt) continue;
      bool same = true;
      for (int t = 0; t <= nt && same; ++t) same = rint[q.rptr + t] == rc[t];
      for (size_t k = 0; k < rcol.size() && same; ++k)
        same = rint[q.ridx + k] == rcol[k] && rdbl[q.rw + k] == rw[k];
      if (same) {
        found = id;
        break;
      }
    }
    if (found >= 0) {
      h->elem_sig[e] = found;
      continue;
    }
    RSig rs{};
    rs.nt = nt;
    // column-compressed form
    std::vector<int> cc(nt + 1, 0);
    for (int col : rcol) cc[col + 1]++;
    for (int t = 0; t < nt; ++t) cc[t + 1] += cc[t];
    std::vector<int> crow(rcol.size());
    std::vector<double> cw(rcol.size());
    std::vector<int> fill(cc.begin(), cc.end() - 1);
    for (int t = 0; t < nt; ++t)
      for (int k = rc[t]; k < rc[t + 1]; ++k) {
        const int dst = fill[rcol[k]]++;
        crow[dst] = t;
        cw[dst] = rw[k];
      }
    rs.cptr = (int64_t)rint.size();
    rint.insert(rint.end(), cc.begin(), cc.end());
    rs.cidx = (int64_t)rint.size();
    rint.insert(rint.end(), crow.begin(), crow.end());
    rs.cw = (int64_t)rdbl.size();
    rdbl.insert(rdbl.end(), cw.begin(), cw.end());
    rs.rptr = (int64_t)rint.size();
    rint.insert(rint.end(), rc.begin(), rc.end());
    rs.ridx = (int64_t)rint.size();
    rint.insert(rint.end(), rcol.begin(), rcol.end());
    rs.rw = (int64_t)rdbl.size();
    rdbl.insert(rdbl.end(), rw.begin(), rw.end());
    const int id = (int)h->rsig.size();
    h->rsig.push_back(rs);
    sig_by_hash[hsh].push_back(id);
    h->elem_sig[e] = id;
  }

  // ---- colouring: elements that touch a common global entity (directly or
  // through a hanging constraint) get different colours ----------------------
  {
    std::vector<std::vector<int>> ent_el(n_ent);
    for (int e = 0; e < ne; ++e)
      for (int en : elem_ents[e]) ent_el[en].push_back(e);
    std::vector<int> color(ne, -1);
    int ncol = 0;
    std::vector<int> mark;
    for (int e = 0; e < ne; ++e) {
      mark.assign(ncol + 1, 0);
      for (int en : elem_ents[e])
        for (int o2 : ent_el[en])
          if (color[o2] >= 0) mark[color[o2]] = 1;
      int c = 0;
      while (c < ncol && mark[c]) ++c;
      color[e] = c;
      if (c == ncol) ++ncol;
    }
    // per group: its elements sorted by colour
    h->ncolor = ncol;
    h->elem_color = color;
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
  for (int e = 0; e < ne; ++e)
    for (int en : elem_ents[e]) ent_elems[en].push_back(e);
  h->blk.clear();
  h->blk_colptr.clear();
  h->cols.clear();
  std::vector<int64_t> rowptr(nfree + 1, 0);
  std::vector<int32_t> row2blk(nfree, -1);
  for (int en = 0; en < n_ent; ++en) {
    const int dE = startE[en] >= 0 ? ent_dofs(en) : 0, dH = startH[en] >= 0 ? ent_dofs(en) : 0;
    if (dE + dH == 0) continue;
    std::vector<int> nb;
    for (int e : ent_elems[en]) nb.insert(nb.end(), elem_ents[e].begin(), elem_ents[e].end());
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
  h->stream = (prm->flags & DPG_FLAG_STREAM) != 0;
  DPG_ALLOC(h->d_off, sizeof(ElemOff) * (ne + 1));
  if (h->stream)
    DPG_ALLOC(h->d_soff, sizeof(ElemOff) * (ne + 1));  // filled with the launch plan
  else
    h->d_soff = h->d_off;
  DPG_ALLOC(h->d_l2g, sizeof(int32_t) * tot.h);
  DPG_ALLOC(h->d_xfix, sizeof(double2) * tot.h);
  DPG_ALLOC(h->d_robin, sizeof(dpg_robin_group) * std::max<size_t>(1, h->robin.size()));
  DPG_ALLOC(h->d_status, sizeof(int) * (ne + 1));  // [ne]: tensor-core wait timeout flag
  if (h->stream && (prm->flags & DPG_FLAG_ADJOINT)) {
    h->err = "DPG_FLAG_STREAM does not keep the factors the adjoint needs (DPG_FLAG_ADJOINT)";
    return DPG_ERR_UNSUPPORTED;
  }
  if (!h->stream) {  // streaming allocates chunk-sized stores with the workspace
    DPG_ALLOC(h->d_S, sizeof(double2) * tot.S);
    DPG_ALLOC(h->d_s, sizeof(double2) * tot.h);
    DPG_ALLOC(h->d_Z, sizeof(double2) * tot.Z);
    DPG_ALLOC(h->d_z, sizeof(double2) * tot.u);
  }
  DPG_ALLOC(h->d_c, sizeof(double) * ne);
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
