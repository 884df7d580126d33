// Host-side structural analysis of the bus/branch graph: done once per grid.
//
// Everything here is integer graph work (orderings, symbolic factorisation,
// level schedules, a depth-first numbering).  No floating-point value of the
// method is computed on the host.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace gpcg {

struct Csr {
  int n = 0;
  std::vector<int32_t> ptr, idx;
  int nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

// Bus adjacency: for bus b, neighbours adj.idx[adj.ptr[b]..] and the branch
// joining them in adj_branch at the same positions.
struct BusGraph {
  Csr adj;
  std::vector<int32_t> adj_branch;
};

// Structure of one fast-decoupled matrix (B' or B'') and of its factor,
// rows numbered in the final solve order (level-sorted).
struct MatrixPlan {
  int n = 0;                          // rows
  std::vector<int32_t> bus_of_row;    // [n]
  std::vector<int32_t> row_of_bus;    // [n_bus], -1 if the bus has no row
  Csr A;                              // full symmetric pattern, cols sorted
  std::vector<int32_t> a_diag;        // [n] position of the diagonal in A
  Csr L;                              // lower pattern, cols sorted, diag last
  Csr U;                              // L^T as rows (diag first), cols sorted
  std::vector<int32_t> l_to_u;        // [nnz(L)] position of L_ij in U
  std::vector<int32_t> level;         // [n] forward level of each row
  std::vector<int32_t> lev_ptr;       // rows of level k: [lev_ptr[k], lev_ptr[k+1])
  std::vector<int32_t> blev_ptr;      // backward levels: positions into blev_rows
  std::vector<int32_t> blev_rows;
  // tail of the forward schedule (see plan_tail): levels [tail_lev, nlev),
  // rows [tail_row0, n); and the backward levels of the rows before it
  int tail_lev = 0, tail_row0 = 0;
  std::vector<int32_t> tblev_ptr, tblev_rows;
};

// Build the bus adjacency from the branch list.
BusGraph build_bus_graph(int n_bus, int n_branch, const int32_t* f, const int32_t* t);

// Plan for the grounded Laplacian on the buses with keep[b] != 0, using the
// given factor pattern: fill = false gives IC(0) (pattern of tril(A)),
// fill = true the complete symbolic Cholesky pattern.  Ordering: minimum
// degree, then rows sorted by forward level.
MatrixPlan plan_matrix(int n_bus, const BusGraph& g, const std::vector<uint8_t>& keep,
                       bool fill);

// Split off the tail of the forward level schedule: the longest run of
// final levels with at most max_rows rows together (none if that is a
// single level).  The rows of a tail only depend, in the backward solve, on
// rows of the tail, so both substitutions of the tail can be done at once
// after the forward levels before it; the backward schedule of the
// remaining rows (tblev_*) treats the tail rows as solved.
void plan_tail(MatrixPlan& P, int max_rows);

// Reverse Cuthill-McKee order of the bus graph (new position -> bus): buses
// adjacent in the grid get nearby positions.
std::vector<int32_t> rcm_order(int n, const BusGraph& g);

// Depth-first numbering from `root`: pre[b] (preorder) and size[b]
// (subtree size).  Returns false when some bus is unreachable.  bridge[l]
// is set for branches whose removal disconnects the graph.
bool dfs_numbering(int n_bus, const BusGraph& g, int root, std::vector<int32_t>& pre,
                   std::vector<int32_t>& size, std::vector<uint8_t>& bridge, int n_branch);

}  // namespace gpcg
