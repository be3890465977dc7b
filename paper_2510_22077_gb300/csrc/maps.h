// Integer maps of the domain decomposition (Sec. 3.2.1-3.2.2, Sec. 4), built on the host once per
// context.  See maps.cpp for the rules.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "stencil.cuh"

namespace pns {

struct Maps {
  std::vector<uint8_t> flags;             // per cell, see stencil.cuh
  std::vector<int> label;                 // per cell: the input pore label (0 on solid)
  std::vector<int> pins;                  // ascending
  std::vector<int> cell_prim;             // per cell: primary grid or -1
  std::vector<int> cell_iface;            // per cell: contact interface or -1
  std::vector<int> face_class;            // per (axis, cell): primary grid, -1 f face, -2 not an unknown
  std::vector<int> owner;                 // per full index: primary grid, -1 interface cell, -3 f face, -2 none
  int n_prim = 0, n_iface = 0, n_dropped = 0;
  std::vector<std::vector<int>> iface_cells;  // cells of each interface (ascending)
  std::vector<std::vector<int>> C;            // interfaces adjacent to each primary grid (ascending)
  std::vector<int> coarse_ifaces;             // interfaces adjacent to some primary grid (ascending)
  std::vector<int> coarse_of_iface;           // coarse index of each interface, -1 if none
  std::vector<std::vector<int>> prim_unk;     // full indices of each primary grid (ascending)
  std::vector<std::vector<int>> dual_unk;     // full indices of each dual grid (ascending)
  long long n_unknowns = 0, n_faces = 0, n_cells = 0;
};

// Returns 0 on success; on bad input fills `err` and returns a negative status.
int build_maps(const Geo& G, const uint8_t* mask, const int32_t* labels, int n_dilate, int n_tag, Maps& M,
               std::string& err);

}  // namespace pns
