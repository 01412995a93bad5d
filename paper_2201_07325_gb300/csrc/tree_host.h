// Host-side description of the octree (built on the GPU by tree.cu).
#pragma once

#include <cuda_runtime.h>
#include <map>
#include <stdint.h>
#include <string>
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
  std::vector<HBox> boxes;         // ids ordered by (level, Morton)
  int nlevels = 0;
  int leaf_size = 64;
  std::map<int, HLevel> levels;    // l >= 2
};

// Builds the whole tree on the GPU (tree.cu) from device points (N x 3
// row-major) and fills T; *d_perm receives a device copy of the sorted
// permutation (cudaFree by the caller). Returns 0 or a negative FMMLU_ERR_*
// code with a message. verbose: phase times (cumulative ms) on stderr.
int gpu_build_tree(const double* pts, int64_t n, int leaf_size, TreeHost& T, int** d_perm,
                   std::string& msg, int verbose, cudaStream_t st);
std::vector<int> current_boxes(const TreeHost& T, int level);

}  // namespace fmmlu
