// blocks.h -- host description of the blocks of every smoother (Sec. 3):
// chains of straight segments plus at most one junction node.  Built in
// closed form by setup.cu; consumed by its work-list packer.
#pragma once
#include <vector>

namespace tmg {

// A segment: len nodes from (i0, j0) in direction dir (DIR_*).  The first
// node of a chain's next segment is this segment's last node plus one step in
// the next segment's direction.
struct HSeg {
  int i0, j0, dir, len;
};
struct HChain {
  std::vector<HSeg> s;
  bool fj = false, lj = false;
  int ljdir = 0;  // direction from the last node to the junction
};
struct HBlock {
  bool junc = false;
  int ji = 0, jj = 0;
  std::vector<HChain> ch;
  int nodes = 0, chunks = 0;
  int group = 0, pos = 0;  // packing order: blocks of one group in order of pos are
                           // neighbours (adjacent same-colour legs / lines)
};

// The blocks of one colour (0 = red, relaxed first) of each line smoother.
void tweed_blocks(int nx, int ny, int colour, std::vector<HBlock> &out);
void wireframe_blocks(int nx, int ny, int colour, std::vector<HBlock> &out);
void zebra_blocks(int nx, int ny, int colour, bool along_x, std::vector<HBlock> &out);

}  // namespace tmg
