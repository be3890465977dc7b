// Domain-decomposition maps (Sec. 3.2.1-3.2.2 and Sec. 4 of the paper).
//
// Rules (the paper leaves these details open; the same rules are stated in the design notes):
//  * unknowns: face (d, c) iff c and c - e_d exist and are void; cell c iff void.
//  * pressure pin: the lowest-index cell of every face-connected void component (periodic wrap).
//  * contact-interface cell: void cell of label a with a face-neighbour of label b > a; its pair is
//    (a, smallest such b).  One interface per pair (Gamma_ij of the paper): all interface cells with
//    that pair, connected or not, numbered by their lowest cell index.
//  * primary grid of label a: its non-interface cells; surviving labels numbered in ascending order.
//  * face class: the primary grid of a flanking cell (never two different ones), else f.
//  * C^{p_i}: interfaces owning a cell face-adjacent to a cell of p_i.
//  * coarse interfaces: those in some C^{p_i}.  An interface adjacent to no primary grid (3D junctions)
//    has no shape vector; a coarse unknown for it would make the coarse matrix singular.
//  * dual grid j: interface j's cells dilated n_dilate times (default 1) over void face-neighbours;
//    unknowns are its cells and every face unknown with a flanking cell in it.
//  * gPLMM tags: f faces, plus primary faces with a same-axis neighbour face (along any axis) that is
//    an unknown of another class; n_tag > 1 repeats with "neighbour is tagged".
#include "maps.h"

#include <algorithm>
#include <climits>
#include <deque>
#include <map>

namespace pns {

int build_maps(const Geo& G, const uint8_t* mask, const int32_t* labels, int n_dilate, int n_tag, Maps& M,
               std::string& err) {
  const int nc = G.ncell, dim = G.dim;
  const long long nfull = (long long)(dim + 1) * nc;
  M.flags.assign(nc, 0);
  M.label.assign(labels, labels + nc);
  for (int c = 0; c < nc; ++c) {
    bool v = mask[c] != 0;
    if (v && labels[c] < 1) { err = "labels must be >= 1 on void cells"; return -1; }
    if (!v && labels[c] != 0) { err = "labels must be 0 on solid cells"; return -1; }
    if (v) M.flags[c] |= FL_VOID;
  }
  for (int c = 0; c < nc; ++c) {
    if (!(M.flags[c] & FL_VOID)) continue;
    for (int d = 0; d < dim; ++d) {
      int lo = nbr_c(G, c, d, -1);
      if (lo >= 0 && (M.flags[lo] & FL_VOID)) M.flags[c] |= fl_face(d);
    }
  }
  auto is_void = [&](int c) { return c >= 0 && (M.flags[c] & FL_VOID); };
  M.n_cells = 0;
  M.n_faces = 0;
  for (int c = 0; c < nc; ++c) {
    if (M.flags[c] & FL_VOID) M.n_cells++;
    for (int d = 0; d < dim; ++d)
      if (M.flags[c] & fl_face(d)) M.n_faces++;
  }
  M.n_unknowns = M.n_cells + M.n_faces;

  // ---- pins
  {
    std::vector<char> seen(nc, 0);
    std::vector<int> q;
    M.pins.clear();
    for (int s = 0; s < nc; ++s) {
      if (!is_void(s) || seen[s]) continue;
      M.pins.push_back(s);
      seen[s] = 1;
      q.assign(1, s);
      for (size_t h = 0; h < q.size(); ++h) {
        int c = q[h];
        CellPos p = cell_pos(G, c);
        for (int a = 0; a < dim; ++a)
          for (int sgn = -1; sgn <= 1; sgn += 2) {
            int n = nbr(G, p, a, sgn);
            if (is_void(n) && !seen[n]) { seen[n] = 1; q.push_back(n); }
          }
      }
    }
    for (int c : M.pins) M.flags[c] |= FL_PIN;
  }

  // ---- interface cells
  std::vector<int> partner(nc, INT_MAX);
  for (int c = 0; c < nc; ++c) {
    if (!is_void(c)) continue;
    CellPos p = cell_pos(G, c);
    for (int a = 0; a < dim; ++a)
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        int n = nbr(G, p, a, sgn);
        if (is_void(n) && labels[n] > labels[c]) partner[c] = std::min(partner[c], (int)labels[n]);
      }
  }
  M.cell_iface.assign(nc, -1);
  M.iface_cells.clear();
  {
    // one interface per label pair, numbered by its lowest cell (cells visited in ascending order)
    std::map<std::pair<int, int>, int> pair_id;
    for (int c = 0; c < nc; ++c) {
      if (partner[c] == INT_MAX) continue;
      auto key = std::make_pair((int)labels[c], partner[c]);
      auto it = pair_id.find(key);
      int id;
      if (it == pair_id.end()) {
        id = (int)M.iface_cells.size();
        pair_id.emplace(key, id);
        M.iface_cells.emplace_back();
      } else {
        id = it->second;
      }
      M.cell_iface[c] = id;
      M.iface_cells[id].push_back(c);
    }
  }
  M.n_iface = (int)M.iface_cells.size();

  // ---- primary grids
  std::map<int, int> lab2p;
  std::map<int, int> all_labels;
  for (int c = 0; c < nc; ++c) {
    if (!is_void(c)) continue;
    all_labels[labels[c]] = 1;
    if (M.cell_iface[c] < 0) lab2p[labels[c]] = 0;
  }
  {
    int k = 0;
    for (auto& kv : lab2p) kv.second = k++;
  }
  M.n_prim = (int)lab2p.size();
  M.n_dropped = (int)(all_labels.size() - lab2p.size());
  M.cell_prim.assign(nc, -1);
  for (int c = 0; c < nc; ++c)
    if (is_void(c) && M.cell_iface[c] < 0) M.cell_prim[c] = lab2p[labels[c]];

  // ---- face classes
  M.face_class.assign((size_t)dim * nc, -2);
  for (int d = 0; d < dim; ++d)
    for (int c = 0; c < nc; ++c) {
      if (!(M.flags[c] & fl_face(d))) continue;
      int lo = nbr_c(G, c, d, -1);
      int pl = M.cell_prim[lo], ph = M.cell_prim[c];
      if (pl >= 0 && ph >= 0 && pl != ph) { err = "a face is flanked by two different primary grids"; return -1; }
      M.face_class[(size_t)d * nc + c] = ph >= 0 ? ph : (pl >= 0 ? pl : -1);
    }

  // ---- C^{p_i}
  M.C.assign(M.n_prim, {});
  for (int c = 0; c < nc; ++c) {
    int j = M.cell_iface[c];
    if (j < 0) continue;
    CellPos p = cell_pos(G, c);
    for (int a = 0; a < dim; ++a)
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        int n = nbr(G, p, a, sgn);
        if (n >= 0 && M.cell_prim[n] >= 0) M.C[M.cell_prim[n]].push_back(j);
      }
  }
  for (auto& v : M.C) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  M.coarse_of_iface.assign(M.n_iface, -1);
  for (auto& v : M.C)
    for (int j : v) M.coarse_of_iface[j] = 0;
  M.coarse_ifaces.clear();
  for (int j = 0; j < M.n_iface; ++j)
    if (M.coarse_of_iface[j] == 0) {
      M.coarse_of_iface[j] = (int)M.coarse_ifaces.size();
      M.coarse_ifaces.push_back(j);
    }

  // ---- owners and primary unknown lists (ascending full index)
  M.owner.assign(nfull, -2);
  for (int d = 0; d < dim; ++d)
    for (int c = 0; c < nc; ++c) {
      int fc = M.face_class[(size_t)d * nc + c];
      if (fc == -2) continue;
      M.owner[(size_t)d * nc + c] = fc >= 0 ? fc : -3;
    }
  for (int c = 0; c < nc; ++c) {
    if (!is_void(c)) continue;
    M.owner[(size_t)dim * nc + c] = M.cell_prim[c] >= 0 ? M.cell_prim[c] : -1;
  }
  M.prim_unk.assign(M.n_prim, {});
  for (long long g = 0; g < nfull; ++g)
    if (M.owner[g] >= 0) M.prim_unk[M.owner[g]].push_back((int)g);

  // ---- dual grids
  M.dual_unk.assign(M.n_iface, {});
  {
    std::vector<int> stamp(nc, -1), fstamp((size_t)dim * nc, -1);
    std::vector<int> cells, frontier, next;
    for (int j = 0; j < M.n_iface; ++j) {
      cells = M.iface_cells[j];
      for (int c : cells) stamp[c] = j;
      frontier = cells;
      for (int it = 0; it < n_dilate; ++it) {
        next.clear();
        for (int c : frontier) {
          CellPos p = cell_pos(G, c);
          for (int a = 0; a < dim; ++a)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
              int n = nbr(G, p, a, sgn);
              if (is_void(n) && stamp[n] != j) { stamp[n] = j; next.push_back(n); }
            }
        }
        cells.insert(cells.end(), next.begin(), next.end());
        frontier.swap(next);
      }
      std::vector<int>& U = M.dual_unk[j];
      for (int c : cells) {
        U.push_back(dim * nc + c);
        for (int d = 0; d < dim; ++d) {
          if ((M.flags[c] & fl_face(d)) && fstamp[(size_t)d * nc + c] != j) {
            fstamp[(size_t)d * nc + c] = j;
            U.push_back(d * nc + c);
          }
          int hi = nbr_c(G, c, d, +1);
          if (face_unknown(M.flags.data(), d, hi) && fstamp[(size_t)d * nc + hi] != j) {
            fstamp[(size_t)d * nc + hi] = j;
            U.push_back(d * nc + hi);
          }
        }
      }
      std::sort(U.begin(), U.end());
    }
  }

  // ---- gPLMM tags
  {
    std::vector<char> tag((size_t)dim * nc, 0), nxt;
    for (int d = 0; d < dim; ++d)
      for (int c = 0; c < nc; ++c) {
        int cls = M.face_class[(size_t)d * nc + c];
        if (cls == -2) continue;
        if (cls == -1) { tag[(size_t)d * nc + c] = 1; continue; }
        CellPos p = cell_pos(G, c);
        for (int a = 0; a < dim; ++a)
          for (int sgn = -1; sgn <= 1; sgn += 2) {
            int n = nbr(G, p, a, sgn);
            if (face_unknown(M.flags.data(), d, n) && M.face_class[(size_t)d * nc + n] != cls) tag[(size_t)d * nc + c] = 1;
          }
      }
    for (int it = 1; it < n_tag; ++it) {
      nxt = tag;
      for (int d = 0; d < dim; ++d)
        for (int c = 0; c < nc; ++c) {
          int cls = M.face_class[(size_t)d * nc + c];
          if (cls < 0) continue;
          CellPos p = cell_pos(G, c);
          for (int a = 0; a < dim; ++a)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
              int n = nbr(G, p, a, sgn);
              if (face_unknown(M.flags.data(), d, n) && tag[(size_t)d * nc + n]) nxt[(size_t)d * nc + c] = 1;
            }
        }
      tag.swap(nxt);
    }
    for (int d = 0; d < dim; ++d)
      for (int c = 0; c < nc; ++c)
        if (tag[(size_t)d * nc + c]) M.flags[c] |= fl_tag(d);
  }
  return 0;
}

}  // namespace pns
