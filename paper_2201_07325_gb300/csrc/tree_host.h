// Host-side octree description (built from GPU-sorted Morton keys).
#pragma once

#include <map>
#include <stdint.h>
#include <unordered_map>
#include <vector>

namespace fmmlu {

struct HBox {
  int level = 0;
  int64_t cx = 0, cy = 0, cz = 0;  // cell at its level
  int64_t start = 0, end = 0;      // sorted point range
  int parent = -1;
  std::vector<int> kids;           // ascending ids (Morton order)
  bool leaf() const { return kids.empty(); }
  int64_t count() const { return end - start; }
};

struct HLevel {
  int level = 0;
  std::vector<int> boxes;          // level boxes (ids, Morton order)
  std::vector<int> current;        // current boxes ordered by point start
  std::vector<int> nbeg, ncnt, nlist;   // per level box (index r): N (box ids)
  std::vector<int> qbeg, qcnt, qlist;   // per level box: Q (box ids)
  std::vector<int> colour;         // per level box
  std::vector<int> order;          // elimination order (indices r)
  int ncolours = 0;
};

struct TreeHost {
  int64_t n = 0;
  double corner[3] = {0, 0, 0};
  double side = 1.0;
  std::vector<int> perm;           // sorted position -> caller index
  std::vector<uint64_t> keys;      // sorted Morton keys
  std::vector<HBox> boxes;
  int nlevels = 0;
  int leaf_size = 64;
  std::map<int, HLevel> levels;    // l >= 2
  std::unordered_map<uint64_t, int> where;   // (level, cell) -> id
};

void build_host_tree(TreeHost& T, int leaf_size);
HLevel build_level(const TreeHost& T, int level);
std::vector<int> current_boxes(const TreeHost& T, int level);
int64_t box_gap(const HBox& a, const HBox& b);
uint64_t morton3_host(int64_t cx, int64_t cy, int64_t cz);

}  // namespace fmmlu
