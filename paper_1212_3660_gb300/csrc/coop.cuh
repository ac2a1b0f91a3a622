// Cooperative V-cycle of the lower multigrid levels: one launch runs every
// phase of levels lc .. coarsest (half sweeps, residual and restriction, the
// coarsest dense solve, interpolation) on the levels' global vectors, with the
// per-cell arithmetic of the per-level kernels, as one thread-block cluster
// per source (levels of at most 65536 cells) or one cooperative grid.
#pragma once
#include "common.cuh"

namespace fks {

template <typename T>
struct CoopParams {
  int nlev;                         // levels lc .. coarsest
  LevelView<T> L[MAX_LEVELS];       // coefficients (global memory)
  const cx<T>* invd[MAX_LEVELS];    // [n_tau][n] inverse diagonals
  cx<T>* f[MAX_LEVELS];             // right-hand sides, slot stride n
  cx<T>* z[MAX_LEVELS];             // iterates, slot stride n
  int rx[MAX_LEVELS], ry[MAX_LEVELS], rz[MAX_LEVELS];
  const cx<T>* Ainv;                // [n_tau][nc][nc] coarsest inverses
  int nc;
  uint32_t mask;
  const z64* taus;
  int nslot;
};

// Positive when either form can be launched on the current device (0: neither).
template <typename T>
int coop_capacity_vcycle();

// Launches the lower V-cycle: one cluster per source, or a cooperative grid of
// `blocks` blocks (at most what can be resident); false when the launch was
// refused.
template <typename T>
bool launch_coop_vcycle(const CoopParams<T>& P, const SlotState* st, int blocks, cudaStream_t s);

}  // namespace fks
