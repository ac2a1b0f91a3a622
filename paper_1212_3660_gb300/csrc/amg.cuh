// Smoothed-aggregation algebraic multigrid for K + tau M (amg.cu): the host
// setup of one tau's hierarchy and the V-cycle that preconditions the BiCGSTAB
// steps of a CSR operator's inner solve (Section 6).
#pragma once
#include <string>
#include <vector>

#include "common.cuh"

namespace fks {

constexpr int AMG_MAX_LEVELS = 16;
constexpr int64_t AMG_MAX_DENSE = 4096;  // largest coarsest level (dense inverse)

// One level of one tau's hierarchy on the device, values in the cycle precision T.
template <typename T>
struct AmgLevel {
  int64_t n, nc;                  // unknowns of this level and of the next (0 on the coarsest)
  const int64_t* arp;             // A_l (level 0: K + tau M on the entries where K or M is nonzero)
  const int32_t* aci;
  const cx<T>* av;
  const cx<T>* dinv;              // 1 / diag(A_l)
  T omega;                        // Jacobi weight 4 / (3 rho_l)
  const int64_t* prp;             // P_l, n x nc
  const int32_t* pci;
  const cx<T>* pv;
  const int64_t* rrp;             // R_l = P_l^T, nc x n
  const int32_t* rci;
  const cx<T>* rv;
  const cx<T>* cinv;              // coarsest level: dense inverse, row-major n x n
};

// ---------------------------------------------------------------- host setup
struct AmgCsr {                   // complex128 CSR, columns sorted within a row
  int64_t n = 0, m = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<z64> v;
};

struct AmgHostLevel {
  AmgCsr A, P, R;
  std::vector<z64> dinv;
  double omega = 0.0;
};

struct AmgHost {
  std::vector<AmgHostLevel> lv;
  std::vector<z64> cinv;          // dense inverse of the coarsest A (row-major)
};

// Aggregates of every level but the coarsest. They depend on the sparsity
// pattern only, so the first tau's build fixes them for every other tau.
struct AmgAgg {
  std::vector<std::vector<int32_t>> agg;
  std::vector<int32_t> count;
};

// The hierarchy of A0 (level 0; its pattern is the strength graph). With
// agg->agg empty the aggregates are computed and stored; otherwise they are
// reused and fix the number of levels. Returns "" or an error message.
std::string amg_build(const AmgCsr& A0, int max_levels, int64_t max_coarse, AmgAgg* agg, AmgHost* out);

// Device copies of a host hierarchy in precision T: every allocation is
// appended to `mem` (the caller frees them, also after an error), one
// AmgLevel per level to `levels`.
template <typename T>
cudaError_t amg_upload(const AmgHost& h, std::vector<void*>& mem, std::vector<AmgLevel<T>>& levels);

// ---------------------------------------------------------------- V-cycle
// Per-level work vectors of a batch ([nslot][n_l] each, cycle precision) and
// the device table of the batch's hierarchies: tab[tau * L + l].
template <typename T>
struct AmgRun {
  const AmgLevel<T>* tab;
  int L, nu;
  int64_t n[AMG_MAX_LEVELS];
  cx<T>* f[AMG_MAX_LEVELS];       // right-hand side of level l >= 1
  cx<T>* x[AMG_MAX_LEVELS];       // iterate
  cx<T>* y[AMG_MAX_LEVELS];       // second Jacobi buffer
  cx<T>* r[AMG_MAX_LEVELS];       // residual, then (l >= 1) the level's result
};

struct BcgScal;
struct SlotState;

// out0 = V_0(f0) for every slot whose inner solve runs and whose BiCGSTAB
// cycle has not halted (sc may be null); returns the number of launches.
template <typename T>
int launch_amg_vcycle(const AmgRun<T>& R, const SlotState* st, const BcgScal* sc, const cx<T>* f0, cx<T>* out0,
                      int nslot, cudaStream_t s);

}  // namespace fks
